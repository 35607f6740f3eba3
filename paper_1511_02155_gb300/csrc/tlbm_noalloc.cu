// tlbm_noalloc.cu -- tlbm_step_noalloc: one time step of the split kernels
// (moments, wetting ghosts, collide + stream, FP64 mass totals) on caller-owned
// population buffers, with every intermediate array held in a fixed-size
// file-scope __device__ buffer instead of memory the library allocates.
//
// It exists for callers that may not allocate device memory at all: code that
// runs inside a host framework which owns every device allocation through its
// own pool, code that must not add allocation latency or fragmentation to a
// time-critical loop, and code that runs where an allocation would be illegal
// (a region being captured into a CUDA graph).  Such callers bring their own
// input and output buffers; this entry point only launches kernels.
//
// The scratch buffers below exist once per device for the life of the process
// (every GPU that loads the library holds them until exit), and all calls share
// them: two calls whose kernels overlap on the GPU (different streams, or the
// same lattice stepped from two host threads) race on the scratch and give
// wrong results.  Serialise calls, e.g. by issuing them on one stream.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/tlbm.h"
#include "tlbm_kernels.cuh"

namespace {

// Moment arrays: 3 * Np values of the compute type (Np = nodes rounded up to 64).
constexpr size_t kScratchBytes = size_t(8) << 20;  // 8 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static __device__ __align__(256) double g_partials[3 * tlbm_dev::kMassBlocks];
static __device__ __align__(256) int g_flag[1];

struct DevPtrs {
    void* scratch;
    double* partials;
    int* flag;
};

std::mutex g_mu;
DevPtrs g_ptrs[kMaxDevices];
bool g_ready[kMaxDevices];
thread_local char g_msg[256];

tlbm_status err(tlbm_status s, const char* what) {
    snprintf(g_msg, sizeof g_msg, "%s", what);
    return s;
}

// Device addresses of the file-scope buffers for the current device.  Host code
// only sees host-side stand-ins for g_scratch & co., so the addresses must come
// from cudaGetSymbolAddress with that device current.  Done once per device.
tlbm_status device_ptrs(DevPtrs* out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(TLBM_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return err(TLBM_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ready[dev]) {
        DevPtrs p{};
        e = cudaGetSymbolAddress(&p.scratch, g_scratch);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&p.partials, g_partials);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&p.flag, g_flag);
        if (e != cudaSuccess) return err(TLBM_ERR_CUDA, cudaGetErrorString(e));
        g_ptrs[dev] = p;
        g_ready[dev] = true;
    }
    *out = g_ptrs[dev];
    return TLBM_OK;
}

template <typename T>
tlbm_dev::Phys<T> phys(const double kappa[3], double alpha, double tau_f, double M_phi, double M_psi,
                       const double h[3]) {
    tlbm_dev::Phys<T> p;
    const double k1 = kappa[0], k2 = kappa[1], k3 = kappa[2], a2 = alpha * alpha;
    for (int m = 0; m < 3; ++m) p.kappa[m] = T(kappa[m]);
    p.a2 = T(a2);
    p.omega[0] = T(1.0 / tau_f);
    p.omega[1] = T(1.0 / (0.5 + M_phi));  // Gamma_phi = 1
    p.omega[2] = T(1.0 / (0.5 + M_psi));  // Gamma_psi = 1
    p.gamma[0] = T(1);
    p.gamma[1] = T(1);
    const double q1 = h[0] / (a2 * k1), q2 = h[1] / (a2 * k2), q3 = h[2] / (a2 * k3);
    p.Gw[0] = T(-q1 - q2 - q3);
    p.Gw[1] = T(-q1 + q2);
    p.Gw[2] = T(-q3);
    const double K[3][3] = {{(k1 + k2) / 4, (k1 - k2) / 4, -(k1 + k2) / 4},
                            {(k1 - k2) / 4, (k1 + k2) / 4, -(k1 - k2) / 4},
                            {-(k1 + k2) / 4, -(k1 - k2) / 4, (k1 + k2 + 4 * k3) / 4}};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) p.K[a][b] = T(K[a][b]);
    return p;
}

template <int Q, typename S>
cudaError_t launch(const tlbm_dev::Geom& g, const tlbm_dev::Phys<typename tlbm_dev::Store<S>::T>& P,
                   const uint8_t* solid, const S* src, S* dst, double* mass, const DevPtrs& sp,
                   cudaStream_t st) {
    using namespace tlbm_dev;
    using T = typename Store<S>::T;
    T* mom = static_cast<T*>(sp.scratch);
    long long b = (g.N + kThreads - 1) / kThreads;
    const int grid = (int)(b < 1 ? 1 : (b > 152LL * 8 ? 152LL * 8 : b));
    if (solid) {
        k_moments<Q, S, true, true><<<kMassBlocks, kThreads, 0, st>>>(g, src, solid, mom, sp.partials);
        k_ghosts<Q, T><<<grid, kThreads, 0, st>>>(g, solid, mom, P);
        k_collide_split<Q, S, true><<<grid, kThreads, 0, st>>>(g, src, dst, solid, mom, P);
    } else {
        k_moments<Q, S, false, true><<<kMassBlocks, kThreads, 0, st>>>(g, src, solid, mom, sp.partials);
        k_collide_split<Q, S, false><<<grid, kThreads, 0, st>>>(g, src, dst, solid, mom, P);
    }
    if (mass) k_mass_final<<<1, kThreads, 0, st>>>(sp.partials, kMassBlocks, mass, sp.flag);
    return cudaGetLastError();
}

}  // namespace

extern "C" tlbm_status tlbm_step_noalloc(tlbm_lattice lattice, tlbm_precision precision, int nx, int ny,
                                         int nz, const double kappa[3], double alpha, double tau_f,
                                         double M_phi, double M_psi, const double h[3],
                                         const uint8_t* solid_dev, const void* src_dev, void* dst_dev,
                                         double* mass_dev, void* cuda_stream) {
    g_msg[0] = '\0';
    if (lattice != TLBM_D2Q9 && lattice != TLBM_D3Q19) return err(TLBM_ERR_ARG, "lattice must be D2Q9 or D3Q19");
    if (nx < 1 || ny < 1 || nz < 1 || (lattice == TLBM_D2Q9 && nz != 1)) return err(TLBM_ERR_ARG, "bad sizes");
    if (!kappa || !src_dev || !dst_dev || src_dev == dst_dev)
        return err(TLBM_ERR_ARG, "kappa, src and dst are required and src != dst");
    if (precision != TLBM_FP32 && precision != TLBM_FP64)
        return err(TLBM_ERR_UNSUPPORTED, "only TLBM_FP32 and TLBM_FP64 storage");
    double hh[3] = {0, 0, 0};
    if (h) for (int m = 0; m < 3; ++m) hh[m] = h[m];
    if (!(alpha > 0) || !(tau_f > 0.5) || !(M_phi > 0) || !(M_psi > 0)) return err(TLBM_ERR_PARAM, "bad parameters");
    for (int m = 0; m < 3; ++m)
        if (!(kappa[m] > 0) || !(std::fabs(4.0 * hh[m] / (alpha * kappa[m])) < 1.0))
            return err(TLBM_ERR_PARAM, "kappa must be > 0 and |4 h/(alpha kappa)| < 1");
    const long long N = (long long)nx * ny * nz;
    const long long Np = (N + 63) / 64 * 64;
    const size_t tsize = precision == TLBM_FP64 ? 8 : 4;
    if ((size_t)Np * 3 * tsize > kScratchBytes)
        return err(TLBM_ERR_ARG, precision == TLBM_FP64
                                     ? "lattice too large for the fixed scratch (at most 349504 nodes in FP64)"
                                     : "lattice too large for the fixed scratch (at most 699008 nodes in FP32)");
    DevPtrs sp;
    tlbm_status s = device_ptrs(&sp);
    if (s != TLBM_OK) return s;
    const tlbm_dev::Geom g{nx, ny, nz, N, Np, (nx + 31) / 32};
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e;
    if (precision == TLBM_FP64) {
        const auto P = phys<double>(kappa, alpha, tau_f, M_phi, M_psi, hh);
        e = lattice == TLBM_D2Q9
                ? launch<9, double>(g, P, solid_dev, (const double*)src_dev, (double*)dst_dev, mass_dev, sp, st)
                : launch<19, double>(g, P, solid_dev, (const double*)src_dev, (double*)dst_dev, mass_dev, sp, st);
    } else {
        const auto P = phys<float>(kappa, alpha, tau_f, M_phi, M_psi, hh);
        e = lattice == TLBM_D2Q9
                ? launch<9, float>(g, P, solid_dev, (const float*)src_dev, (float*)dst_dev, mass_dev, sp, st)
                : launch<19, float>(g, P, solid_dev, (const float*)src_dev, (float*)dst_dev, mass_dev, sp, st);
    }
    if (e != cudaSuccess) return err(TLBM_ERR_CUDA, cudaGetErrorString(e));
    return TLBM_OK;
}

extern "C" const char* tlbm_noalloc_last_error(void) { return g_msg; }
