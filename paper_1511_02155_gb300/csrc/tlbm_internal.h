// tlbm_internal.h -- host-side structures shared by the C ABI (tlbm_api.cu)
// and the per-precision kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tlbm_host {

// Physical parameters in double; each translation unit converts to its compute type.
struct PhysD {
    double kappa[3];
    double a2;        // alpha^2
    double omega[3];  // 1/tau_f, 1/tau_phi, 1/tau_psi
    double gamma[2];  // Gamma_phi, Gamma_psi
    double Gw[3];     // wall-normal gradients of rho, phi, psi
    double K[3][3];   // mixing coefficients kappa_XY
};

// Blocks of the fixed grid of the split step's moment/mass kernels and of
// tlbm_mass.  Fixed (not derived from the device) so that the FP64 totals are
// summed in the same order, hence bitwise the same, on every GPU.
constexpr int kMassBlocks = 1216;

// Physical parameters of the step from the ABI's arguments (Gamma_phi,
// Gamma_psi = 1 unless set): relaxation rates, wall-normal gradients of the
// wetting condition and the pressure tensor's mixing coefficients.  One helper
// for the engine and the allocation-free step.
PhysD make_phys(const double kappa[3], double alpha, double tau_f, double M_phi, double M_psi,
                const double gamma[2], const double h[3]);

enum Kind { KIND_FUSED = 1, KIND_SPLIT = 2 };

struct DevState {
    int Q;
    int prec;            // tlbm_precision
    int nx, ny, nz;
    long long N, Np;     // nodes; stride of node-indexed moment arrays
    int ncx;             // 32-node chunks per row of the population layout
    long long pop_bytes; // bytes of one population buffer
    void* pop[2];        // A-B population buffers (chunk layout, see tlbm_lattice.cuh)
    int cur;             // buffer holding the current state
    const uint8_t* solid;  // device mask (nullptr when there are no solid nodes)
    uint32_t* nbm;       // per-node neighbour-solid bits for the fused step (with solids)
    int nbm_ready;       // nbm has been built
    void* mom;           // split-step moment arrays [3][Np] (compute type); scratch
    double* partials;    // mass partial sums, 3 per block
    double* step_mass;   // [3] totals accumulated inside the last step
    double* mass_tmp;    // [3] totals of tlbm_mass
    int* flag;           // non-finite flag (int)
    PhysD phys;
    int tile;            // fused-kernel tile choice (0 = default)
    int sms;             // multiprocessors of the device (sizes the fused grid's chunks)
    unsigned long long* check;  // device word: first bounds violation of a checked step
    int checked;         // 1: the fused step runs its bounds-checked kernels
    long long partials_cap;  // blocks whose partial sums fit in the first part of partials
    int coupling;        // 0: pressure-tensor equilibrium; 1: forcing (Guo) coupling
    void* aux;           // forcing coupling's node arrays [NA][Np] (compute type)
};

// A batch of engines of one lattice and storage format, advanced together by
// one launch per step.
struct BatchState {
    int count;
    DevState** sims;     // member engines' device states
    void* desc;          // device descriptor array: [2][count], one set per buffer parity
    int tile;            // tile choice for every member (DevState::tile encoding)
    long long blocks;    // blocks of one batched step
    int built;           // descriptors are current
};

// Buffers of one adjoint run (all device memory, allocated by the caller).
struct AdjJob {
    long long nsteps;     // forward steps from the initial equilibrium
    int K;                // checkpoint interval
    size_t state_bytes;   // bytes of one population state
    const double* target; // [N] target C_3
    void* ckpt;           // ceil(nsteps / K) states: x(0), x(K), ...
    void* seg;            // min(K, nsteps) states: one recomputed segment
    void* fin;            // x(nsteps), restored at the end
    void* lam[2];         // adjoint states (population layout)
    double* work;         // dX[3], dJ[3], dG[9], dLap[3] node arrays (18 Np values of the compute type)
    double* partials;     // 3 doubles per block of the fixed grid
    double* acc;          // [0] loss, [1..3] dL/dkappa (local part), [4..6] dL/dG_X
    double* dfields;      // [3][N] dL/d(rho, phi, psi) of the initial fields
};

struct Ops {
    // one time step; flips cur.  When ev0/ev1 are not null they are recorded on
    // the stream just before and just after the step's main kernel(s).
    cudaError_t (*step)(DevState& d, int kind, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1);
    // populations at equilibrium of device double fields (u may be nullptr)
    cudaError_t (*init)(DevState& d, const double* rho, const double* phi, const double* psi,
                        const double* u, cudaStream_t st);
    cudaError_t (*fields)(DevState& d, double* C1, double* C2, double* C3, double* rho, double* u,
                          cudaStream_t st);
    cudaError_t (*mass)(DevState& d, double* out, cudaStream_t st);
    cudaError_t (*get_box)(DevState& d, int x0, int y0, int z0, int bx, int by, int bz, double* out,
                           cudaStream_t st);
    cudaError_t (*set_pops)(DevState& d, const double* in, cudaStream_t st);
    int (*launches)(const DevState& d, int kind);
    // compute-type values per node of the forcing coupling's node arrays
    int (*aux_per_node)();
    bool (*has_fused)(const DevState& d);
    // batches: build the descriptors of both parities (and neighbour masks);
    // one step of every member (flips every member's cur)
    cudaError_t (*batch_build)(BatchState& b, cudaStream_t st);
    // one batched step of every member; ev0/ev1 (if not null) bracket the main kernel
    cudaError_t (*batch_step)(BatchState& b, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1);
    // forward run with checkpoints, then the adjoint back to the initial fields
    // (FP64 and FP32 storage; cudaErrorNotSupported for the 16-bit formats)
    cudaError_t (*adjoint)(DevState& d, int kind, const AdjJob& job, cudaStream_t st);
};

// one table per storage format and lattice (one translation unit each)
const Ops* ops_fp64_q9();
const Ops* ops_fp64_q19();
const Ops* ops_fp32_q9();
const Ops* ops_fp32_q19();
const Ops* ops_fp16_q9();
const Ops* ops_fp16_q19();
const Ops* ops_bf16_q9();
const Ops* ops_bf16_q19();

// the table of a storage format (tlbm_precision) and lattice (Q); nullptr if not built
const Ops* ops_for(int precision, int Q);

int mass_blocks();

}  // namespace tlbm_host
