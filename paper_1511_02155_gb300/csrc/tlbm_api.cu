// tlbm_api.cu -- the C ABI declared in include/tlbm.h: parameter checks,
// device memory, host<->device copies, and dispatch to the kernel tables of
// each storage format.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tlbm.h"
#include "tlbm_internal.h"

using tlbm_host::DevState;
using tlbm_host::Ops;

struct tlbm {
    DevState d;
    const Ops* ops;
    cudaStream_t st;
    int device;
    int kind_req;          // tlbm_kernel requested
    int64_t steps;
    int rest_init;         // state is the u = 0 equilibrium set by tlbm_init_fields (no step since)
    double kappa[3], alpha, tau_f, M_phi, M_psi, gamma[2], h[3];
    size_t esize;          // bytes per stored population
    size_t tsize;          // bytes per compute value
    double* staging;       // device doubles for init/fields (8 N), allocated on demand
    size_t partials_len;   // doubles in d.partials
    cudaEvent_t ev[2];     // kernel timing events (timing mode)
    int timing;            // 1: time the main kernel(s) of every step
    double kernel_ms;      // accumulated main-kernel time in timing mode
    int64_t kernel_steps;  // steps accumulated in kernel_ms
    std::string err;
};

namespace {

thread_local std::string g_create_err;

tlbm_status fail(tlbm* t, tlbm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (t) t->err = buf;
    else g_create_err = buf;
    return s;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(t, e_ == cudaErrorMemoryAllocation ? TLBM_ERR_OOM : TLBM_ERR_CUDA,      \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                      \
    } while (0)

void set_phys(tlbm* t) {
    t->d.phys = tlbm_host::make_phys(t->kappa, t->alpha, t->tau_f, t->M_phi, t->M_psi, t->gamma, t->h);
}

int resolve_kind(const tlbm* t) {
    if (t->kind_req == TLBM_KERNEL_SPLIT) return tlbm_host::KIND_SPLIT;
    if (t->kind_req == TLBM_KERNEL_FUSED) return tlbm_host::KIND_FUSED;
    return t->ops->has_fused(t->d) ? tlbm_host::KIND_FUSED : tlbm_host::KIND_SPLIT;
}

tlbm_status ensure_staging(tlbm* t) {
    if (t->staging) return TLBM_OK;
    CK(cudaMalloc(&t->staging, sizeof(double) * 8 * (size_t)t->d.N));
    return TLBM_OK;
}

tlbm_status ensure_mom(tlbm* t) {
    if (t->d.mom) return TLBM_OK;
    CK(cudaMalloc(&t->d.mom, t->tsize * 3 * (size_t)t->d.Np));
    return TLBM_OK;
}

}  // namespace

namespace tlbm_host {
int mass_blocks() { return kMassBlocks; }

PhysD make_phys(const double kappa[3], double alpha, double tau_f, double M_phi, double M_psi,
                const double gamma[2], const double h[3]) {
    PhysD p{};
    const double k1 = kappa[0], k2 = kappa[1], k3 = kappa[2];
    for (int m = 0; m < 3; ++m) p.kappa[m] = kappa[m];
    p.a2 = alpha * alpha;
    // BGK rates: tau_phi = 1/2 + M_phi / Gamma_phi, tau_psi likewise (Eqs. Mobility1/2)
    p.omega[0] = 1.0 / tau_f;
    p.omega[1] = 1.0 / (0.5 + M_phi / gamma[0]);
    p.omega[2] = 1.0 / (0.5 + M_psi / gamma[1]);
    p.gamma[0] = gamma[0];
    p.gamma[1] = gamma[1];
    // wall-normal gradients of rho, phi, psi (wetting conditions on the auxiliary fields)
    const double q1 = h[0] / (p.a2 * k1), q2 = h[1] / (p.a2 * k2), q3 = h[2] / (p.a2 * k3);
    p.Gw[0] = -q1 - q2 - q3;
    p.Gw[1] = -q1 + q2;
    p.Gw[2] = -q3;
    // mixing coefficients of the pressure tensor
    p.K[0][0] = (k1 + k2) / 4.0;
    p.K[1][1] = (k1 + k2) / 4.0;
    p.K[2][2] = (k1 + k2 + 4.0 * k3) / 4.0;
    p.K[0][1] = p.K[1][0] = (k1 - k2) / 4.0;
    p.K[1][2] = p.K[2][1] = -(k1 - k2) / 4.0;
    p.K[0][2] = p.K[2][0] = -(k1 + k2) / 4.0;
    return p;
}

const Ops* ops_for(int precision, int Q) {
    if (Q != 9 && Q != 19) return nullptr;
    const bool q9 = Q == 9;
    switch (precision) {
        case TLBM_FP64: return q9 ? ops_fp64_q9() : ops_fp64_q19();
        case TLBM_FP32: return q9 ? ops_fp32_q9() : ops_fp32_q19();
        case TLBM_FP16_OFFSET: return q9 ? ops_fp16_q9() : ops_fp16_q19();
        case TLBM_BF16_OFFSET: return q9 ? ops_bf16_q9() : ops_bf16_q19();
    }
    return nullptr;
}
}  // namespace tlbm_host

extern "C" {

const char* tlbm_status_string(tlbm_status s) {
    switch (s) {
        case TLBM_OK: return "TLBM_OK";
        case TLBM_ERR_ARG: return "TLBM_ERR_ARG";
        case TLBM_ERR_PARAM: return "TLBM_ERR_PARAM";
        case TLBM_ERR_CUDA: return "TLBM_ERR_CUDA";
        case TLBM_ERR_OOM: return "TLBM_ERR_OOM";
        case TLBM_ERR_NONFINITE: return "TLBM_ERR_NONFINITE";
        case TLBM_ERR_TIMEOUT: return "TLBM_ERR_TIMEOUT";
        case TLBM_ERR_UNSUPPORTED: return "TLBM_ERR_UNSUPPORTED";
    }
    return "TLBM_ERR_UNKNOWN";
}

const char* tlbm_last_error(const tlbm* t) {
    if (!t) return g_create_err.c_str();
    return t->err.c_str();
}

void tlbm_destroy(tlbm* t) {
    if (!t) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(t->device);
    if (t->st) cudaStreamSynchronize(t->st);
    else cudaDeviceSynchronize();
    cudaFree(t->d.pop[0]);
    cudaFree(t->d.pop[1]);
    cudaFree((void*)t->d.solid);
    cudaFree(t->d.nbm);
    cudaFree(t->d.mom);
    cudaFree(t->d.aux);
    cudaFree(t->d.partials);
    cudaFree(t->d.step_mass);
    cudaFree(t->d.mass_tmp);
    cudaFree(t->d.flag);
    cudaFree(t->d.check);
    cudaFree(t->staging);
    if (t->ev[0]) cudaEventDestroy(t->ev[0]);
    if (t->ev[1]) cudaEventDestroy(t->ev[1]);
    if (prev >= 0) cudaSetDevice(prev);
    delete t;
}

tlbm_status tlbm_create(tlbm** out, tlbm_lattice lattice, int nx, int ny, int nz, const double kappa[3],
                        double alpha, double tau_f, double M_phi, double M_psi, const double h[3],
                        const uint8_t* solid_mask, tlbm_precision precision, void* cuda_stream) {
    tlbm* t = nullptr;
    g_create_err.clear();
    if (!out) return fail(nullptr, TLBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (lattice != TLBM_D2Q9 && lattice != TLBM_D3Q19)
        return fail(nullptr, TLBM_ERR_ARG, "lattice must be TLBM_D2Q9 or TLBM_D3Q19");
    if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, TLBM_ERR_ARG, "sizes must be >= 1");
    if (lattice == TLBM_D2Q9 && nz != 1) return fail(nullptr, TLBM_ERR_ARG, "D2Q9 needs nz == 1");
    if (!kappa) return fail(nullptr, TLBM_ERR_ARG, "kappa is NULL");
    const long long N = (long long)nx * ny * nz;
    if (N > (1LL << 40)) return fail(nullptr, TLBM_ERR_ARG, "lattice too large");
    double hh[3] = {0, 0, 0};
    if (h) for (int m = 0; m < 3; ++m) hh[m] = h[m];
    if (!(alpha > 0) || !std::isfinite(alpha)) return fail(nullptr, TLBM_ERR_PARAM, "alpha must be > 0");
    for (int m = 0; m < 3; ++m) {
        if (!(kappa[m] > 0) || !std::isfinite(kappa[m]))
            return fail(nullptr, TLBM_ERR_PARAM, "kappa_%d must be > 0", m + 1);
        if (!std::isfinite(hh[m]) || !(std::fabs(4.0 * hh[m] / (alpha * kappa[m])) < 1.0))
            return fail(nullptr, TLBM_ERR_PARAM, "|4 h_%d / (alpha kappa_%d)| must be < 1", m + 1, m + 1);
    }
    if (!(tau_f > 0.5) || !std::isfinite(tau_f)) return fail(nullptr, TLBM_ERR_PARAM, "tau_f must be > 1/2");
    if (!(M_phi > 0) || !(M_psi > 0) || !std::isfinite(M_phi) || !std::isfinite(M_psi))
        return fail(nullptr, TLBM_ERR_PARAM, "mobilities must be > 0");
    const Ops* ops = nullptr;
    size_t esize = 0, tsize = 0;
    switch (precision) {
        case TLBM_FP64: esize = 8; tsize = 8; break;
        case TLBM_FP32: esize = 4; tsize = 4; break;
        case TLBM_FP16_OFFSET: esize = 2; tsize = 4; break;
        case TLBM_BF16_OFFSET: esize = 2; tsize = 4; break;
        default: return fail(nullptr, TLBM_ERR_ARG, "unknown precision");
    }
    ops = tlbm_host::ops_for(precision, lattice);
    if (!ops) return fail(nullptr, TLBM_ERR_UNSUPPORTED, "precision/lattice combination not built");

    t = new tlbm();
    memset(&t->d, 0, sizeof t->d);
    t->ops = ops;
    t->st = static_cast<cudaStream_t>(cuda_stream);
    t->kind_req = TLBM_KERNEL_AUTO;
    t->steps = 0;
    for (int m = 0; m < 3; ++m) { t->kappa[m] = kappa[m]; t->h[m] = hh[m]; }
    t->alpha = alpha; t->tau_f = tau_f; t->M_phi = M_phi; t->M_psi = M_psi;
    t->gamma[0] = t->gamma[1] = 1.0;
    t->esize = esize; t->tsize = tsize;
    t->staging = nullptr;
    t->ev[0] = t->ev[1] = nullptr;
    t->timing = 0;
    t->kernel_ms = 0.0;
    t->kernel_steps = 0;
    cudaGetDevice(&t->device);
    DevState& d = t->d;
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, t->device) != cudaSuccess || d.sms < 1) {
        cudaGetLastError();  // not sticky; the allocations below report a missing device
        d.sms = 1;
    }
    d.Q = (int)lattice; d.prec = (int)precision;
    d.nx = nx; d.ny = ny; d.nz = nz; d.N = N;
    d.Np = (N + 63) / 64 * 64;
    d.ncx = (nx + 31) / 32;
    // bytes of one 32-node chunk (see the layout notes in tlbm_lattice.cuh): FP64
    // and D2Q9 FP32 all 3Q populations; D3Q19 FP32 3(Q-1)/2 runs of two-value
    // lane words for the moving populations and two for the rest populations
    // (one value unused); 16-bit formats 3(Q-1)/2 runs of 16-bit pairs and three
    // FP32 rest runs
    const long long chunk = esize == 2   ? (long long)((d.Q - 1) + (d.Q - 1) / 2 + 3) * 128
                            : esize == 4 && d.Q == 19 ? (long long)((d.Q - 1) + (d.Q - 1) / 2 + 2) * 256
                                         : 3LL * d.Q * 32 * (long long)esize;
    d.pop_bytes = (long long)ny * nz * d.ncx * chunk;
    d.cur = 0;
    d.tile = 0;
    set_phys(t);

    auto bail = [&](tlbm_status s) {
        g_create_err = t->err;
        tlbm_destroy(t);
        return s;
    };
    const size_t popbytes = (size_t)d.pop_bytes;
    for (int b = 0; b < 2; ++b) {
        cudaError_t e = cudaMalloc(&d.pop[b], popbytes);
        if (e != cudaSuccess)
            return bail(fail(t, TLBM_ERR_OOM, "cudaMalloc(%zu bytes) for populations: %s", popbytes,
                             cudaGetErrorString(e)));
        e = cudaMemsetAsync(d.pop[b], 0, popbytes, t->st);
        if (e != cudaSuccess) return bail(fail(t, TLBM_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e)));
    }
    bool any_solid = false;
    if (solid_mask)
        for (long long r = 0; r < N && !any_solid; ++r) any_solid = solid_mask[r] != 0;
    if (any_solid) {
        uint8_t* ds = nullptr;
        cudaError_t e = cudaMalloc(&ds, (size_t)N);
        if (e != cudaSuccess) return bail(fail(t, TLBM_ERR_OOM, "cudaMalloc(mask): %s", cudaGetErrorString(e)));
        d.solid = ds;
        e = cudaMemcpy(ds, solid_mask, (size_t)N, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return bail(fail(t, TLBM_ERR_CUDA, "cudaMemcpy(mask): %s", cudaGetErrorString(e)));
        // neighbour-solid bits of the fused step, built by its first launch
        e = cudaMalloc(&d.nbm, sizeof(uint32_t) * (size_t)N);
        if (e != cudaSuccess) return bail(fail(t, TLBM_ERR_OOM, "cudaMalloc(neighbour mask): %s", cudaGetErrorString(e)));
        d.nbm_ready = 0;
    }
    // mass partials: step partials (up to one per fused block) + tlbm_mass partials
    long long nblk = 0;
    {
        // generous bound on fused blocks: one per 64 nodes
        nblk = N / 64 + 1;
        if (nblk < tlbm_host::mass_blocks()) nblk = tlbm_host::mass_blocks();
    }
    t->partials_len = 3 * (size_t)(nblk + tlbm_host::mass_blocks());
    d.partials_cap = nblk;
    cudaError_t e = cudaMalloc(&d.partials, sizeof(double) * t->partials_len);
    if (e == cudaSuccess) e = cudaMalloc(&d.step_mass, sizeof(double) * 3);
    if (e == cudaSuccess) e = cudaMalloc(&d.mass_tmp, sizeof(double) * 3);
    if (e == cudaSuccess) e = cudaMalloc(&d.flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&d.check, sizeof(unsigned long long));
    if (e != cudaSuccess) return bail(fail(t, TLBM_ERR_OOM, "cudaMalloc(reductions): %s", cudaGetErrorString(e)));
    const double nan3[3] = {NAN, NAN, NAN};
    e = cudaMemcpy(d.step_mass, nan3, sizeof nan3, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d.flag, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d.check, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaStreamSynchronize(t->st);
    if (e != cudaSuccess) return bail(fail(t, TLBM_ERR_CUDA, "initialisation: %s", cudaGetErrorString(e)));
    *out = t;
    return TLBM_OK;
}

tlbm_status tlbm_set_gamma(tlbm* t, double gamma_phi, double gamma_psi) {
    if (!t) return TLBM_ERR_ARG;
    if (!(gamma_phi > 0) || !(gamma_psi > 0)) return fail(t, TLBM_ERR_PARAM, "Gamma must be > 0");
    t->gamma[0] = gamma_phi;
    t->gamma[1] = gamma_psi;
    set_phys(t);
    return TLBM_OK;
}

tlbm_status tlbm_set_kernel(tlbm* t, tlbm_kernel kind) {
    if (!t) return TLBM_ERR_ARG;
    if (kind != TLBM_KERNEL_AUTO && kind != TLBM_KERNEL_FUSED && kind != TLBM_KERNEL_SPLIT)
        return fail(t, TLBM_ERR_ARG, "unknown kernel kind");
    if (kind == TLBM_KERNEL_FUSED && !t->ops->has_fused(t->d))
        return fail(t, TLBM_ERR_UNSUPPORTED, "fused step not available for this configuration");
    t->kind_req = kind;
    return TLBM_OK;
}

tlbm_kernel tlbm_get_kernel(const tlbm* t) {
    if (!t) return TLBM_KERNEL_AUTO;
    return resolve_kind(t) == tlbm_host::KIND_FUSED ? TLBM_KERNEL_FUSED : TLBM_KERNEL_SPLIT;
}

// Tile choice of the fused step: variant (0 = default) and planes per chunk (0 = auto).
tlbm_status tlbm_set_tile(tlbm* t, int variant, int chunk) {
    if (!t) return TLBM_ERR_ARG;
    if (variant < 0 || variant > 255 || (variant & 15) > 7 || chunk < 0 || chunk > 4096)
        return fail(t, TLBM_ERR_ARG, "bad tile");
    t->d.tile = variant + 256 * chunk;
    // partial sums must fit: blocks grow as chunks shrink
    return TLBM_OK;
}

tlbm_status tlbm_set_coupling(tlbm* t, tlbm_coupling coupling) {
    if (!t) return TLBM_ERR_ARG;
    if (coupling != TLBM_COUPLING_PRESSURE_TENSOR && coupling != TLBM_COUPLING_FORCING)
        return fail(t, TLBM_ERR_ARG, "unknown coupling");
    if (coupling == TLBM_COUPLING_FORCING) {
        if (t->d.solid)
            return fail(t, TLBM_ERR_UNSUPPORTED, "the forcing coupling runs on lattices without solid nodes");
        tlbm_status s = ensure_mom(t);
        if (s != TLBM_OK) return s;
        if (!t->d.aux)
            CK(cudaMalloc(&t->d.aux, t->tsize * (size_t)t->ops->aux_per_node() * (size_t)t->d.Np));
    }
    t->d.coupling = coupling == TLBM_COUPLING_FORCING ? 1 : 0;
    return TLBM_OK;
}

tlbm_coupling tlbm_get_coupling(const tlbm* t) {
    return t && t->d.coupling ? TLBM_COUPLING_FORCING : TLBM_COUPLING_PRESSURE_TENSOR;
}

tlbm_status tlbm_set_bounds_check(tlbm* t, int on) {
    if (!t) return TLBM_ERR_ARG;
    if (on && t->d.prec != TLBM_FP32)
        return fail(t, TLBM_ERR_UNSUPPORTED, "bounds-checked kernels exist for TLBM_FP32 storage only");
    t->d.checked = on ? 1 : 0;
    return TLBM_OK;
}

tlbm_status tlbm_bounds_check_word(tlbm* t, uint64_t* word) {
    if (!t || !word) return TLBM_ERR_ARG;
    unsigned long long w = 0;
    CK(cudaStreamSynchronize(t->st));
    CK(cudaMemcpy(&w, t->d.check, sizeof w, cudaMemcpyDeviceToHost));
    if (w) CK(cudaMemset(t->d.check, 0, sizeof w));
    *word = (uint64_t)w;
    return TLBM_OK;
}

tlbm_status tlbm_init_fields(tlbm* t, const double* rho, const double* phi, const double* psi,
                             const double* ux, const double* uy, const double* uz) {
    if (!t) return TLBM_ERR_ARG;
    if (!rho || !phi || !psi) return fail(t, TLBM_ERR_ARG, "rho, phi, psi must not be NULL");
    tlbm_status s = ensure_staging(t);
    if (s != TLBM_OK) return s;
    s = ensure_mom(t);
    if (s != TLBM_OK) return s;
    const size_t N = (size_t)t->d.N, nb = N * sizeof(double);
    double* st = t->staging;
    CK(cudaMemcpyAsync(st, rho, nb, cudaMemcpyHostToDevice, t->st));
    CK(cudaMemcpyAsync(st + N, phi, nb, cudaMemcpyHostToDevice, t->st));
    CK(cudaMemcpyAsync(st + 2 * N, psi, nb, cudaMemcpyHostToDevice, t->st));
    const double* du = nullptr;
    if (ux || uy || uz) {
        double* u = st + 3 * N;
        if (ux) CK(cudaMemcpyAsync(u, ux, nb, cudaMemcpyHostToDevice, t->st));
        else CK(cudaMemsetAsync(u, 0, nb, t->st));
        if (uy) CK(cudaMemcpyAsync(u + N, uy, nb, cudaMemcpyHostToDevice, t->st));
        else CK(cudaMemsetAsync(u + N, 0, nb, t->st));
        if (uz) CK(cudaMemcpyAsync(u + 2 * N, uz, nb, cudaMemcpyHostToDevice, t->st));
        else CK(cudaMemsetAsync(u + 2 * N, 0, nb, t->st));
        du = u;
    }
    CK(t->ops->init(t->d, st, st + N, st + 2 * N, du, t->st));
    CK(cudaMemsetAsync(t->d.flag, 0, sizeof(int), t->st));
    CK(cudaStreamSynchronize(t->st));
    t->steps = 0;
    t->rest_init = du == nullptr ? 1 : 0;
    return TLBM_OK;
}

tlbm_status tlbm_step(tlbm* t, int64_t nsteps) {
    if (!t) return TLBM_ERR_ARG;
    if (nsteps < 0) return fail(t, TLBM_ERR_ARG, "nsteps must be >= 0");
    const int kind = resolve_kind(t);
    if (kind == tlbm_host::KIND_SPLIT) {
        tlbm_status s = ensure_mom(t);
        if (s != TLBM_OK) return s;
    }
    for (int64_t n = 0; n < nsteps; ++n) {
        if (t->timing) {
            CK(t->ops->step(t->d, kind, t->st, t->ev[0], t->ev[1]));
            float ms = 0.0f;
            CK(cudaEventSynchronize(t->ev[1]));
            CK(cudaEventElapsedTime(&ms, t->ev[0], t->ev[1]));
            t->kernel_ms += ms;
            ++t->kernel_steps;
        } else {
            CK(t->ops->step(t->d, kind, t->st, nullptr, nullptr));
        }
        ++t->steps;
    }
    return TLBM_OK;
}

int64_t tlbm_steps_done(const tlbm* t) { return t ? t->steps : -1; }

tlbm_status tlbm_set_timing(tlbm* t, int on) {
    if (!t) return TLBM_ERR_ARG;
    if (on && !t->ev[0]) {
        CK(cudaEventCreate(&t->ev[0]));
        CK(cudaEventCreate(&t->ev[1]));
    }
    t->timing = on ? 1 : 0;
    t->kernel_ms = 0.0;
    t->kernel_steps = 0;
    return TLBM_OK;
}

tlbm_status tlbm_kernel_time(const tlbm* t, double* ms_total, int64_t* steps) {
    if (!t || !ms_total || !steps) return TLBM_ERR_ARG;
    *ms_total = t->kernel_ms;
    *steps = t->kernel_steps;
    return TLBM_OK;
}

int tlbm_launches_per_step(const tlbm* t) {
    if (!t) return -1;
    return t->ops->launches(t->d, resolve_kind(t));
}

tlbm_status tlbm_fields(tlbm* t, double* C1, double* C2, double* C3, double* rho, double* u) {
    if (!t) return TLBM_ERR_ARG;
    tlbm_status s = ensure_staging(t);
    if (s != TLBM_OK) return s;
    const size_t N = (size_t)t->d.N, nb = N * sizeof(double);
    double* st = t->staging;
    CK(t->ops->fields(t->d, C1 ? st : nullptr, C2 ? st + N : nullptr, C3 ? st + 2 * N : nullptr,
                      rho ? st + 3 * N : nullptr, u ? st + 4 * N : nullptr, t->st));
    if (C1) CK(cudaMemcpyAsync(C1, st, nb, cudaMemcpyDeviceToHost, t->st));
    if (C2) CK(cudaMemcpyAsync(C2, st + N, nb, cudaMemcpyDeviceToHost, t->st));
    if (C3) CK(cudaMemcpyAsync(C3, st + 2 * N, nb, cudaMemcpyDeviceToHost, t->st));
    if (rho) CK(cudaMemcpyAsync(rho, st + 3 * N, nb, cudaMemcpyDeviceToHost, t->st));
    if (u) CK(cudaMemcpyAsync(u, st + 4 * N, 3 * nb, cudaMemcpyDeviceToHost, t->st));
    CK(cudaStreamSynchronize(t->st));
    return TLBM_OK;
}

tlbm_status tlbm_mass(tlbm* t, double out[3]) {
    if (!t || !out) return TLBM_ERR_ARG;
    CK(t->ops->mass(t->d, t->d.mass_tmp, t->st));
    CK(cudaMemcpyAsync(out, t->d.mass_tmp, 3 * sizeof(double), cudaMemcpyDeviceToHost, t->st));
    CK(cudaStreamSynchronize(t->st));
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(out[c])) return fail(t, TLBM_ERR_NONFINITE, "mass total %d is not finite", c);
    return TLBM_OK;
}

tlbm_status tlbm_step_mass(tlbm* t, double out[3]) {
    if (!t || !out) return TLBM_ERR_ARG;
    int flag = 0;
    CK(cudaMemcpyAsync(out, t->d.step_mass, 3 * sizeof(double), cudaMemcpyDeviceToHost, t->st));
    CK(cudaMemcpyAsync(&flag, t->d.flag, sizeof(int), cudaMemcpyDeviceToHost, t->st));
    CK(cudaStreamSynchronize(t->st));
    if (flag) return fail(t, TLBM_ERR_NONFINITE, "a step produced a non-finite mass total");
    return TLBM_OK;
}

tlbm_status tlbm_get_populations_box(tlbm* t, int x0, int y0, int z0, int bx, int by, int bz,
                                     double* host) {
    if (!t || !host) return TLBM_ERR_ARG;
    if (bx < 1 || by < 1 || bz < 1) return fail(t, TLBM_ERR_ARG, "box sizes must be >= 1");
    const size_t n = 3 * (size_t)t->d.Q * (size_t)bx * by * bz;
    double* dv = nullptr;
    CK(cudaMalloc(&dv, n * sizeof(double)));
    cudaError_t e = t->ops->get_box(t->d, x0, y0, z0, bx, by, bz, dv, t->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, dv, n * sizeof(double), cudaMemcpyDeviceToHost, t->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(t->st);
    cudaFree(dv);
    if (e != cudaSuccess) return fail(t, TLBM_ERR_CUDA, "get_populations_box: %s", cudaGetErrorString(e));
    return TLBM_OK;
}

tlbm_status tlbm_get_populations(tlbm* t, double* host) {
    if (!t) return TLBM_ERR_ARG;
    return tlbm_get_populations_box(t, 0, 0, 0, t->d.nx, t->d.ny, t->d.nz, host);
}

tlbm_status tlbm_set_populations(tlbm* t, const double* host) {
    if (!t || !host) return TLBM_ERR_ARG;
    const size_t n = 3 * (size_t)t->d.Q * (size_t)t->d.N;
    double* dv = nullptr;
    CK(cudaMalloc(&dv, n * sizeof(double)));
    cudaError_t e = cudaMemcpyAsync(dv, host, n * sizeof(double), cudaMemcpyHostToDevice, t->st);
    if (e == cudaSuccess) e = t->ops->set_pops(t->d, dv, t->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->d.flag, 0, sizeof(int), t->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(t->st);
    cudaFree(dv);
    if (e != cudaSuccess) return fail(t, TLBM_ERR_CUDA, "set_populations: %s", cudaGetErrorString(e));
    t->steps = 0;
    t->rest_init = 0;
    return TLBM_OK;
}

size_t tlbm_state_bytes(const tlbm* t) {
    if (!t) return 0;
    return (size_t)t->d.pop_bytes;
}

tlbm_status tlbm_get_state(tlbm* t, void* host, size_t bytes) {
    if (!t || !host) return TLBM_ERR_ARG;
    if (bytes != tlbm_state_bytes(t)) return fail(t, TLBM_ERR_ARG, "state is %zu bytes", tlbm_state_bytes(t));
    CK(cudaMemcpyAsync(host, t->d.pop[t->d.cur], bytes, cudaMemcpyDeviceToHost, t->st));
    CK(cudaStreamSynchronize(t->st));
    return TLBM_OK;
}

tlbm_status tlbm_set_state(tlbm* t, const void* host, size_t bytes) {
    if (!t || !host) return TLBM_ERR_ARG;
    if (bytes != tlbm_state_bytes(t)) return fail(t, TLBM_ERR_ARG, "state is %zu bytes", tlbm_state_bytes(t));
    CK(cudaMemcpyAsync(t->d.pop[t->d.cur], host, bytes, cudaMemcpyHostToDevice, t->st));
    CK(cudaMemsetAsync(t->d.flag, 0, sizeof(int), t->st));
    CK(cudaStreamSynchronize(t->st));
    t->rest_init = 0;
    return TLBM_OK;
}

tlbm_status tlbm_adjoint_c3_misfit(tlbm* t, int64_t nsteps, int checkpoint_every, const double* target,
                                   double* loss, double dkappa[3], double dh[3], double* dfields) {
    if (!t) return TLBM_ERR_ARG;
    if (nsteps < 1 || checkpoint_every < 1) return fail(t, TLBM_ERR_ARG, "nsteps and checkpoint_every must be >= 1");
    if (!target || !loss || !dkappa || !dh) return fail(t, TLBM_ERR_ARG, "target, loss, dkappa and dh are required");
    if (t->d.prec != TLBM_FP64 && t->d.prec != TLBM_FP32)
        return fail(t, TLBM_ERR_UNSUPPORTED, "the adjoint needs TLBM_FP64 or TLBM_FP32 storage");
    if (t->d.coupling)
        return fail(t, TLBM_ERR_UNSUPPORTED, "the adjoint differentiates the pressure-tensor coupling only");
    if (!t->rest_init || t->steps != 0)
        return fail(t, TLBM_ERR_ARG,
                    "the adjoint starts from the state of tlbm_init_fields with u = NULL and no step since");
    tlbm_status s = ensure_mom(t);
    if (s != TLBM_OK) return s;
    const int kind = resolve_kind(t);
    const long long T = nsteps;
    const int K = (int)(checkpoint_every < nsteps ? checkpoint_every : nsteps);
    const long long nseg = (T + K - 1) / K;
    const size_t sb = tlbm_state_bytes(t);
    const size_t N = (size_t)t->d.N, Np = (size_t)t->d.Np;
    const int nblk = tlbm_host::mass_blocks();
    tlbm_host::AdjJob J{};
    J.nsteps = T;
    J.K = K;
    J.state_bytes = sb;
    void* blocks[9] = {};
    const size_t sizes[9] = {sb * (size_t)nseg, sb * (size_t)K, sb, sb, sb, sizeof(double) * 18 * Np,
                             sizeof(double) * 3 * (size_t)nblk, sizeof(double) * 8, sizeof(double) * 4 * N};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 9 && e == cudaSuccess; ++k) e = cudaMalloc(&blocks[k], sizes[k]);
    auto release = [&]() {
        for (void* b : blocks) cudaFree(b);
    };
    if (e != cudaSuccess) {
        release();
        return fail(t, TLBM_ERR_OOM, "adjoint buffers (%zu MB of checkpoints and segment states): %s",
                    (sizes[0] + sizes[1]) >> 20, cudaGetErrorString(e));
    }
    J.ckpt = blocks[0];
    J.seg = blocks[1];
    J.fin = blocks[2];
    J.lam[0] = blocks[3];
    J.lam[1] = blocks[4];
    J.work = static_cast<double*>(blocks[5]);
    J.partials = static_cast<double*>(blocks[6]);
    J.acc = static_cast<double*>(blocks[7]);
    double* tgt = static_cast<double*>(blocks[8]);
    J.target = tgt;
    J.dfields = tgt + N;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    e = cudaMemsetAsync(J.acc, 0, sizeof(double) * 8, t->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tgt, target, sizeof(double) * N, cudaMemcpyHostToDevice, t->st);
    if (e == cudaSuccess) e = t->ops->adjoint(t->d, kind, J, t->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(acc, J.acc, sizeof(double) * 8, cudaMemcpyDeviceToHost, t->st);
    if (e == cudaSuccess && dfields)
        e = cudaMemcpyAsync(dfields, J.dfields, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, t->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(t->st);
    release();
    if (e != cudaSuccess) return fail(t, TLBM_ERR_CUDA, "adjoint run: %s", cudaGetErrorString(e));
    t->steps += nsteps;
    t->rest_init = 0;
    // wall-normal gradients G_X = (-q1 - q2 - q3, -q1 + q2, -q3), q_m = h_m / (alpha^2 kappa_m)
    const double a2 = t->alpha * t->alpha;
    const double dG0 = acc[4], dG1 = acc[5], dG2 = acc[6];
    const double dq[3] = {-dG0 - dG1, -dG0 + dG1, -dG0 - dG2};
    *loss = acc[0];
    for (int m = 0; m < 3; ++m) {
        const double q = t->h[m] / (a2 * t->kappa[m]);
        dh[m] = dq[m] / (a2 * t->kappa[m]);
        dkappa[m] = acc[1 + m] - dq[m] * q / t->kappa[m];
    }
    if (!std::isfinite(*loss)) return fail(t, TLBM_ERR_NONFINITE, "non-finite loss");
    return TLBM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches

struct tlbm_batch {
    tlbm_host::BatchState bs;
    std::vector<tlbm*> members;
    std::vector<DevState*> sims;
    std::vector<tlbm_host::PhysD> phys;  // members' parameters baked into the descriptors
    const Ops* ops;
    cudaStream_t st;       // the members' stream
    cudaStream_t cap;      // private stream used only to capture the step graph
    cudaGraphExec_t exec;  // two batched steps (parity returns to graph_par)
    int graph_par;
    int use_graph;
    cudaEvent_t ev[2];     // main-kernel timing (tlbm_batch_set_timing)
    int timing;
    double kernel_ms;
    int64_t kernel_steps;
    std::string err;
};

namespace {

tlbm_status bfail(tlbm_batch* b, tlbm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    else g_create_err = buf;
    return s;
}

void drop_graph(tlbm_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

tlbm_status batch_rebuild(tlbm_batch* b) {
    drop_graph(b);
    cudaError_t e = b->ops->batch_build(b->bs, b->st);
    if (e != cudaSuccess)
        return bfail(b, e == cudaErrorInvalidConfiguration ? TLBM_ERR_ARG : TLBM_ERR_CUDA,
                     "batch set-up failed: %s", cudaGetErrorString(e));
    b->phys.clear();
    for (DevState* d : b->sims) b->phys.push_back(d->phys);
    return TLBM_OK;
}

// members at one buffer parity, with the parameters the descriptors hold
// (rebuilt when tlbm_set_gamma changed a member since)
tlbm_status batch_aligned(tlbm_batch* b) {
    for (size_t k = 0; k < b->sims.size(); ++k)
        if (b->sims[k]->coupling)
            return bfail(b, TLBM_ERR_UNSUPPORTED, "member %zu uses the forcing coupling (no batched kernel)", k);
    for (size_t k = 1; k < b->sims.size(); ++k)
        if (b->sims[k]->cur != b->sims[0]->cur)
            return bfail(b, TLBM_ERR_ARG, "batch members are at different step parities (a member was stepped alone)");
    bool same = b->phys.size() == b->sims.size();
    for (size_t k = 0; same && k < b->sims.size(); ++k)
        same = memcmp(&b->phys[k], &b->sims[k]->phys, sizeof(tlbm_host::PhysD)) == 0;
    return same ? TLBM_OK : batch_rebuild(b);
}

tlbm_status batch_plain_steps(tlbm_batch* b, int64_t n) {
    for (int64_t k = 0; k < n; ++k) {
        cudaError_t e = b->timing ? b->ops->batch_step(b->bs, b->st, b->ev[0], b->ev[1])
                                  : b->ops->batch_step(b->bs, b->st, nullptr, nullptr);
        if (e == cudaSuccess && b->timing) {
            float ms = 0.0f;
            e = cudaEventSynchronize(b->ev[1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
            b->kernel_ms += ms;
            ++b->kernel_steps;
        }
        if (e != cudaSuccess) return bfail(b, TLBM_ERR_CUDA, "batched step: %s", cudaGetErrorString(e));
        for (tlbm* m : b->members) ++m->steps;
    }
    return TLBM_OK;
}

}  // namespace

extern "C" {

tlbm_status tlbm_batch_create(tlbm_batch** out, tlbm* const* members, int count) {
    g_create_err.clear();
    if (!out || !members || count < 1) return bfail(nullptr, TLBM_ERR_ARG, "need at least one member");
    *out = nullptr;
    for (int k = 0; k < count; ++k) {
        const tlbm* m = members[k];
        if (!m) return bfail(nullptr, TLBM_ERR_ARG, "member %d is NULL", k);
        const tlbm* m0 = members[0];
        if (m->d.Q != m0->d.Q || m->d.prec != m0->d.prec)
            return bfail(nullptr, TLBM_ERR_ARG, "members must share lattice and precision");
        if (m->st != m0->st || m->device != m0->device)
            return bfail(nullptr, TLBM_ERR_ARG, "members must share the device and stream");
        if ((m->d.solid != nullptr) != (m0->d.solid != nullptr))
            return bfail(nullptr, TLBM_ERR_ARG, "members must all have, or all lack, solid nodes");
        if (m->d.coupling)
            return bfail(nullptr, TLBM_ERR_UNSUPPORTED, "member %d uses the forcing coupling (no batched kernel)", k);
        for (int j = 0; j < k; ++j)
            if (members[j] == m) return bfail(nullptr, TLBM_ERR_ARG, "member %d appears twice", k);
    }
    tlbm_batch* b = new tlbm_batch();
    b->members.assign(members, members + count);
    for (tlbm* m : b->members) b->sims.push_back(&m->d);
    b->ops = members[0]->ops;
    b->st = members[0]->st;
    b->cap = nullptr;
    b->exec = nullptr;
    b->graph_par = 0;
    b->use_graph = 0;
    b->ev[0] = b->ev[1] = nullptr;
    b->timing = 0;
    b->kernel_ms = 0.0;
    b->kernel_steps = 0;
    memset(&b->bs, 0, sizeof b->bs);
    b->bs.count = count;
    b->bs.sims = b->sims.data();
    b->bs.tile = 0;
    tlbm_status s = batch_aligned(b);  // first build: no parameters recorded yet
    if (s != TLBM_OK) {
        g_create_err = b->err;
        tlbm_batch_destroy(b);
        return s;
    }
    *out = b;
    return TLBM_OK;
}

void tlbm_batch_destroy(tlbm_batch* b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    else cudaDeviceSynchronize();
    drop_graph(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    cudaFree(b->bs.desc);
    delete b;
}

const char* tlbm_batch_last_error(const tlbm_batch* b) { return b ? b->err.c_str() : g_create_err.c_str(); }

int64_t tlbm_batch_blocks(const tlbm_batch* b) { return b ? (int64_t)b->bs.blocks : -1; }

tlbm_status tlbm_batch_set_tile(tlbm_batch* b, int variant, int chunk) {
    if (!b) return TLBM_ERR_ARG;
    if (variant < 0 || variant > 255 || (variant & 15) > 7 || chunk < 0 || chunk > 4096)
        return bfail(b, TLBM_ERR_ARG, "bad tile");
    const int old = b->bs.tile;
    b->bs.tile = variant + 256 * chunk;
    tlbm_status s = batch_rebuild(b);
    if (s != TLBM_OK) {  // keep the previous, working tile
        b->bs.tile = old;
        batch_rebuild(b);
    }
    return s;
}

tlbm_status tlbm_batch_set_graph(tlbm_batch* b, int on) {
    if (!b) return TLBM_ERR_ARG;
    b->use_graph = on ? 1 : 0;
    if (!on) drop_graph(b);
    return TLBM_OK;
}

tlbm_status tlbm_batch_set_timing(tlbm_batch* b, int on) {
    if (!b) return TLBM_ERR_ARG;
    if (on && !b->ev[0]) {
        if (cudaEventCreate(&b->ev[0]) != cudaSuccess || cudaEventCreate(&b->ev[1]) != cudaSuccess)
            return bfail(b, TLBM_ERR_CUDA, "cudaEventCreate failed");
    }
    b->timing = on ? 1 : 0;
    b->kernel_ms = 0.0;
    b->kernel_steps = 0;
    return TLBM_OK;
}

tlbm_status tlbm_batch_kernel_time(const tlbm_batch* b, double* ms_total, int64_t* steps) {
    if (!b || !ms_total || !steps) return TLBM_ERR_ARG;
    *ms_total = b->kernel_ms;
    *steps = b->kernel_steps;
    return TLBM_OK;
}

tlbm_status tlbm_batch_step(tlbm_batch* b, int64_t nsteps) {
    if (!b) return TLBM_ERR_ARG;
    if (nsteps < 0) return bfail(b, TLBM_ERR_ARG, "nsteps must be >= 0");
    tlbm_status s = batch_aligned(b);
    if (s != TLBM_OK) return s;
    if (!b->use_graph || b->timing || nsteps < 2) return batch_plain_steps(b, nsteps);
    // graph of two batched steps, captured once on a private stream and replayed
    // on the members' stream; it starts and ends at buffer parity graph_par
    if (b->exec && b->sims[0]->cur != b->graph_par) {
        s = batch_plain_steps(b, 1);
        if (s != TLBM_OK) return s;
        --nsteps;
    }
    if (!b->exec) {
        cudaError_t e = cudaSuccess;
        if (!b->cap) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return bfail(b, TLBM_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        const int par = b->sims[0]->cur;
        cudaError_t e1 = b->ops->batch_step(b->bs, b->cap, nullptr, nullptr);
        cudaError_t e2 = b->ops->batch_step(b->bs, b->cap, nullptr, nullptr);  // parity is back to par
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(b->cap, &graph);
        if (e == cudaSuccess && e1 == cudaSuccess && e2 == cudaSuccess)
            e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e == cudaSuccess) e = (e1 != cudaSuccess) ? e1 : e2;
        if (e != cudaSuccess) {
            drop_graph(b);
            return bfail(b, TLBM_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        }
        b->graph_par = par;
    }
    for (int64_t k = 0; k + 1 < nsteps; k += 2) {
        cudaError_t e = cudaGraphLaunch(b->exec, b->st);
        if (e != cudaSuccess) return bfail(b, TLBM_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
        for (tlbm* m : b->members) m->steps += 2;
    }
    return batch_plain_steps(b, nsteps & 1);
}

tlbm_status tlbm_batch_autotune(tlbm_batch* b, int trial_steps, int* variant, int* chunk) {
    if (!b || trial_steps < 1) return TLBM_ERR_ARG;
    tlbm_status s = batch_aligned(b);
    if (s != TLBM_OK) return s;
    const bool solid = b->sims[0]->solid != nullptr;
    const bool d2 = b->sims[0]->Q == 9;
    std::vector<int> shapes = {0};
    if (solid && d2 && b->sims[0]->prec != 0) shapes = {1, 2, 3};
    const int chunks[] = {0, 16, 32, 64};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return bfail(b, TLBM_ERR_CUDA, "cudaEventCreate failed");
    }
    float best = 3.0e38f;
    int bv = 0, bc = 0;
    const int old = b->bs.tile;
    for (int sh : shapes) {
        for (int ch : chunks) {
            b->bs.tile = sh + 256 * ch;
            if (batch_rebuild(b) != TLBM_OK) continue;  // e.g. too many blocks for the partial sums
            if (batch_plain_steps(b, 1) != TLBM_OK) continue;
            cudaEventRecord(e0, b->st);
            if (batch_plain_steps(b, trial_steps) != TLBM_OK) continue;
            cudaEventRecord(e1, b->st);
            float ms = 0.0f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) continue;
            if (ms < best) {
                best = ms;
                bv = sh;
                bc = ch;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->bs.tile = best < 3.0e38f ? bv + 256 * bc : old;
    s = batch_rebuild(b);
    if (s != TLBM_OK) return s;
    if (variant) *variant = bv;
    if (chunk) *chunk = bc;
    return best < 3.0e38f ? TLBM_OK : bfail(b, TLBM_ERR_CUDA, "no tile candidate ran");
}

}  // extern "C"
