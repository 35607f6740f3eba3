// tlbm_noalloc.cu -- tlbm_step_noalloc: one time step of the split kernels
// (moments, wetting ghosts, collide + stream, FP64 mass totals) on caller-owned
// population buffers, with every intermediate array held in a fixed-size
// file-scope __device__ buffer instead of memory the library allocates.
//
// It exists for callers that may not allocate device memory at all: a plug-in
// inside a host framework that owns every device allocation through its own
// pool and budget, where an allocation behind the framework's back would break
// its accounting or fail, and time-critical loops that must not pay allocation
// latency or fragment memory.  Such callers bring their own input and output
// buffers; this entry point only launches the engine's split-step kernels.
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
#include "tlbm_internal.h"

namespace {

// Moment arrays: 3 * Np values of the compute type (Np = nodes rounded up to 64).
constexpr size_t kScratchBytes = size_t(8) << 20;  // 8 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static __device__ __align__(256) double g_partials[3 * tlbm_host::kMassBlocks];
static __device__ __align__(256) double g_mass[3];  // totals when the caller passes no mass_dev
static __device__ __align__(256) int g_flag[1];     // the step's non-finite flag (never read)

struct DevPtrs {
    void* scratch;
    double* partials;
    double* mass;
    int* flag;
    int sms;
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
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&p.mass, g_mass);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&p.flag, g_flag);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return err(TLBM_ERR_CUDA, cudaGetErrorString(e));
        g_ptrs[dev] = p;
        g_ready[dev] = true;
    }
    *out = g_ptrs[dev];
    return TLBM_OK;
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
    // the same parameter checks as tlbm_create
    double hh[3] = {0, 0, 0};
    if (h) for (int m = 0; m < 3; ++m) hh[m] = h[m];
    if (!(alpha > 0) || !std::isfinite(alpha)) return err(TLBM_ERR_PARAM, "alpha must be > 0 and finite");
    if (!(tau_f > 0.5) || !std::isfinite(tau_f)) return err(TLBM_ERR_PARAM, "tau_f must be > 1/2 and finite");
    if (!(M_phi > 0) || !(M_psi > 0) || !std::isfinite(M_phi) || !std::isfinite(M_psi))
        return err(TLBM_ERR_PARAM, "mobilities must be > 0 and finite");
    for (int m = 0; m < 3; ++m)
        if (!(kappa[m] > 0) || !std::isfinite(kappa[m]) || !std::isfinite(hh[m]) ||
            !(std::fabs(4.0 * hh[m] / (alpha * kappa[m])) < 1.0))
            return err(TLBM_ERR_PARAM, "kappa must be > 0 and finite, and |4 h/(alpha kappa)| < 1");
    const long long N = (long long)nx * ny * nz;
    const long long Np = (N + 63) / 64 * 64;
    const size_t tsize = precision == TLBM_FP64 ? 8 : 4;
    if ((size_t)Np * 3 * tsize > kScratchBytes)
        return err(TLBM_ERR_ARG, precision == TLBM_FP64
                                     ? "lattice too large for the fixed scratch (at most 349504 nodes in FP64)"
                                     : "lattice too large for the fixed scratch (at most 699008 nodes in FP32)");
    const tlbm_host::Ops* ops = tlbm_host::ops_for(precision, lattice);
    if (!ops) return err(TLBM_ERR_UNSUPPORTED, "precision/lattice combination not built");
    DevPtrs sp;
    tlbm_status s = device_ptrs(&sp);
    if (s != TLBM_OK) return s;
    // a device state over the caller's buffers and the file-scope scratch; the
    // step is the engine's own split step (same kernels, same parameters)
    tlbm_host::DevState d{};
    d.Q = (int)lattice;
    d.prec = (int)precision;
    d.nx = nx; d.ny = ny; d.nz = nz;
    d.N = N; d.Np = Np;
    d.ncx = (nx + 31) / 32;
    d.pop[0] = const_cast<void*>(src_dev);
    d.pop[1] = dst_dev;
    d.cur = 0;
    d.solid = solid_dev;
    d.mom = sp.scratch;
    d.partials = sp.partials;
    d.step_mass = mass_dev ? mass_dev : sp.mass;
    d.flag = sp.flag;
    const double gamma[2] = {1.0, 1.0};
    d.phys = tlbm_host::make_phys(kappa, alpha, tau_f, M_phi, M_psi, gamma, hh);
    d.sms = sp.sms;
    const cudaError_t e = ops->step(d, tlbm_host::KIND_SPLIT, static_cast<cudaStream_t>(cuda_stream), nullptr, nullptr);
    if (e != cudaSuccess) return err(TLBM_ERR_CUDA, cudaGetErrorString(e));
    return TLBM_OK;
}

extern "C" const char* tlbm_noalloc_last_error(void) { return g_msg; }
