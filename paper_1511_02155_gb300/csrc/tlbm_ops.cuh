// tlbm_ops.cuh -- launch table of one storage format: turns the ABI's device
// state into kernel launches.  Included once per precision translation unit.
#pragma once

#include "tlbm_adjoint.cuh"
#include "tlbm_fused.cuh"
#include "tlbm_guo.cuh"
#include "tlbm_kernels.cuh"

namespace tlbm_dev {

using tlbm_host::DevState;
using tlbm_host::PhysD;

inline Geom geom(const DevState& d) { return Geom{d.nx, d.ny, d.nz, d.N, d.Np, d.ncx}; }

// grid of a grid-stride kernel over n items: at most 8 blocks per SM (the
// results do not depend on the grid)
inline int grid_for(long long n, int sms) {
    long long b = (n + kThreads - 1) / kThreads;
    const long long cap = 8LL * (sms < 1 ? 1 : sms);
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <int Q, typename S>
struct Impl {
    using T = typename Store<S>::T;

    template <bool SOLID>
    static void split(DevState& d, cudaStream_t st) {
        const Geom g = geom(d);
        const Phys<T> P = to_phys<T>(d.phys);
        const S* src = static_cast<const S*>(d.pop[d.cur]);
        S* dst = static_cast<S*>(d.pop[1 - d.cur]);
        T* mom = static_cast<T*>(d.mom);
        const int grid = grid_for(g.N, d.sms);
        k_moments<Q, S, SOLID, true><<<kMassBlocks, kThreads, 0, st>>>(g, src, d.solid, mom, d.partials);
        if (SOLID) k_ghosts<Q, T><<<grid, kThreads, 0, st>>>(g, d.solid, mom, P);
        k_collide_split<Q, S, SOLID><<<grid, kThreads, 0, st>>>(g, src, dst, d.solid, mom, P);
    }

    // moments of src into mom (block partials into part) and the forcing
    // coupling's Pi, mu_phi, mu_psi into aux
    static void guo_aux(DevState& d, const S* src, double* part, cudaStream_t st) {
        const Geom g = geom(d);
        T* mom = static_cast<T*>(d.mom);
        k_moments<Q, S, false, true><<<kMassBlocks, kThreads, 0, st>>>(g, src, nullptr, mom, part);
        k_guo_pressure<Q, T><<<grid_for(g.N, d.sms), kThreads, 0, st>>>(g, mom, static_cast<T*>(d.aux),
                                                                         to_phys<T>(d.phys));
    }

    static void guo(DevState& d, cudaStream_t st) {
        const S* src = static_cast<const S*>(d.pop[d.cur]);
        guo_aux(d, src, d.partials, st);
        const Geom g = geom(d);
        k_guo_collide<Q, S><<<grid_for(g.N, d.sms), kThreads, 0, st>>>(
            g, src, static_cast<S*>(d.pop[1 - d.cur]), static_cast<const T*>(d.aux), to_phys<T>(d.phys));
    }

    static int aux_per_node() { return GuoAux<Q>::NA; }

    static cudaError_t step(DevState& d, int kind, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1) {
        if (ev0) cudaEventRecord(ev0, st);
        if (d.coupling && kind == tlbm_host::KIND_FUSED) {
            cudaError_t e = guo_fused_step<Q, S>(d, to_phys<T>(d.phys), st);
            if (e != cudaSuccess) return e;
        } else if (d.coupling) {
            guo(d, st);
        } else if (kind == tlbm_host::KIND_FUSED) {
            cudaError_t e = fused_step<Q, S>(d, to_phys<T>(d.phys), st);
            if (e != cudaSuccess) return e;
        } else {
            if (d.solid) split<true>(d, st);
            else split<false>(d, st);
        }
        if (ev1) cudaEventRecord(ev1, st);
        k_mass_final<<<1, kThreads, 0, st>>>(d.partials, fused_partials<Q, S>(d, kind), d.step_mass,
                                             d.flag);
        d.cur ^= 1;
        return cudaGetLastError();
    }

    static cudaError_t init(DevState& d, const double* rho, const double* phi, const double* psi,
                            const double* u, cudaStream_t st) {
        const Geom g = geom(d);
        const Phys<T> P = to_phys<T>(d.phys);
        T* mom = static_cast<T*>(d.mom);
        S* dst = static_cast<S*>(d.pop[d.cur]);
        const int grid = grid_for(g.N, d.sms);
        k_fields_to_mom<T><<<grid, kThreads, 0, st>>>(g, rho, phi, psi, d.solid, mom);
        if (d.coupling) {
            T* aux = static_cast<T*>(d.aux);
            k_guo_pressure<Q, T><<<grid, kThreads, 0, st>>>(g, mom, aux, P);
            k_guo_init<Q, S><<<grid, kThreads, 0, st>>>(g, dst, mom, aux, u, P);
        } else if (d.solid) {
            k_ghosts<Q, T><<<grid, kThreads, 0, st>>>(g, d.solid, mom, P);
            k_init_eq<Q, S, true><<<grid, kThreads, 0, st>>>(g, dst, d.solid, mom, u, P);
        } else {
            k_init_eq<Q, S, false><<<grid, kThreads, 0, st>>>(g, dst, d.solid, mom, u, P);
        }
        return cudaGetLastError();
    }

    static cudaError_t fields(DevState& d, double* C1, double* C2, double* C3, double* rho, double* u,
                              cudaStream_t st) {
        const Geom g = geom(d);
        const S* src = static_cast<const S*>(d.pop[d.cur]);
        const int grid = grid_for(g.N, d.sms);
        if (d.solid) k_fields<Q, S, true><<<grid, kThreads, 0, st>>>(g, src, d.solid, C1, C2, C3, rho, u);
        else k_fields<Q, S, false><<<grid, kThreads, 0, st>>>(g, src, d.solid, C1, C2, C3, rho, u);
        if (d.coupling && u) {
            // fluid velocity (j + F/2) / rho of the forcing coupling
            guo_aux(d, src, d.partials + 3 * d.partials_cap, st);
            k_guo_velocity<Q, T><<<grid, kThreads, 0, st>>>(g, static_cast<const T*>(d.mom),
                                                             static_cast<const T*>(d.aux), u);
        }
        return cudaGetLastError();
    }

    static cudaError_t mass(DevState& d, double* out, cudaStream_t st) {
        const Geom g = geom(d);
        const S* src = static_cast<const S*>(d.pop[d.cur]);
        double* part = d.partials + 3 * d.partials_cap;  // after the step partials
        if (d.solid)
            k_moments<Q, S, true, false><<<kMassBlocks, kThreads, 0, st>>>(g, src, d.solid, nullptr, part);
        else
            k_moments<Q, S, false, false><<<kMassBlocks, kThreads, 0, st>>>(g, src, d.solid, nullptr, part);
        k_mass_final<<<1, kThreads, 0, st>>>(part, kMassBlocks, out, d.flag);
        return cudaGetLastError();
    }

    static cudaError_t get_box(DevState& d, int x0, int y0, int z0, int bx, int by, int bz, double* out,
                               cudaStream_t st) {
        const Geom g = geom(d);
        const S* src = static_cast<const S*>(d.pop[d.cur]);
        const int grid = grid_for((long long)bx * by * bz, d.sms);
        if (d.solid)
            k_get_box<Q, S, true><<<grid, kThreads, 0, st>>>(g, src, d.solid, x0, y0, z0, bx, by, bz, out);
        else
            k_get_box<Q, S, false><<<grid, kThreads, 0, st>>>(g, src, d.solid, x0, y0, z0, bx, by, bz, out);
        return cudaGetLastError();
    }

    static cudaError_t set_pops(DevState& d, const double* in, cudaStream_t st) {
        const Geom g = geom(d);
        S* dst = static_cast<S*>(d.pop[d.cur]);
        const int grid = grid_for(g.N, d.sms);
        if (d.solid) k_set_pops<Q, S, true><<<grid, kThreads, 0, st>>>(g, in, d.solid, dst);
        else k_set_pops<Q, S, false><<<grid, kThreads, 0, st>>>(g, in, d.solid, dst);
        return cudaGetLastError();
    }

    static int launches(const DevState& d, int kind) {
        if (kind == tlbm_host::KIND_FUSED) return fused_launches<Q, S>(d) + 1;
        if (d.coupling) return 3 + 1;
        return (d.solid ? 3 : 2) + 1;
    }

    static bool has_fused(const DevState& d) { return fused_supported<Q, S>(d); }

    template <bool SOLID>
    static cudaError_t adjoint_run(DevState& d, int kind, const tlbm_host::AdjJob& J, cudaStream_t st) {
        const Geom g = geom(d);
        const Phys<T> P = to_phys<T>(d.phys);
        T* mom = static_cast<T*>(d.mom);
        const int grid = grid_for(g.N, d.sms);
        const long long Np = g.Np;
        T* wk = reinterpret_cast<T*>(J.work);
        T *dX = wk, *dJ = wk + 3 * Np, *dG = wk + 6 * Np, *dL = wk + 15 * Np;
        auto state = [&](void* base, long long k) { return static_cast<char*>(base) + k * (long long)J.state_bytes; };
        auto cp = [&](void* dst, const void* src) {
            return cudaMemcpyAsync(dst, src, J.state_bytes, cudaMemcpyDeviceToDevice, st);
        };
        cudaError_t e = cudaSuccess;
        auto chk = [&](cudaError_t r) {
            if (e == cudaSuccess && r != cudaSuccess) e = r;
        };
        // moments (with wetting ghosts) of state x into mom
        auto moments_of = [&](const S* x) {
            k_moments<Q, S, SOLID, true><<<kMassBlocks, kThreads, 0, st>>>(g, x, d.solid, mom, d.partials);
            if (SOLID) k_ghosts<Q, T><<<grid, kThreads, 0, st>>>(g, d.solid, mom, P);
        };
        // node adjoint and stencil transpose (the last stage follows at the call site)
        auto adjoint_core = [&](const S* x, const S* lam, auto init_tag) {
            constexpr bool INIT = decltype(init_tag)::value;
            moments_of(x);
            k_adj_node<Q, S, SOLID, INIT><<<kMassBlocks, kThreads, 0, st>>>(g, x, d.solid, mom, lam, P, dX, dJ,
                                                                             dG, dL, J.partials);
            k_adj_acc<<<1, kThreads, 0, st>>>(J.partials, kMassBlocks, 3, J.acc + 1);
            k_adj_gather<Q, T, SOLID><<<kMassBlocks, kThreads, 0, st>>>(g, d.solid, dX, dG, dL, J.partials);
            k_adj_acc<<<1, kThreads, 0, st>>>(J.partials, kMassBlocks, 3, J.acc + 4);
        };
        const long long T = J.nsteps;
        const int K = J.K;
        const long long nseg = (T + K - 1) / K;
        // forward, checkpoints at multiples of K
        chk(cp(state(J.ckpt, 0), d.pop[d.cur]));
        for (long long t = 1; t <= T && e == cudaSuccess; ++t) {
            chk(step(d, kind, st, nullptr, nullptr));
            if (t % K == 0 && t < T) chk(cp(state(J.ckpt, t / K), d.pop[d.cur]));
        }
        const int curT = d.cur;
        chk(cp(J.fin, d.pop[d.cur]));
        // seed: dL/dx(T) of the C_3 misfit
        k_adj_seed<Q, S, SOLID><<<kMassBlocks, kThreads, 0, st>>>(g, static_cast<const S*>(J.fin), d.solid,
                                                                   J.target, static_cast<S*>(J.lam[0]),
                                                                   J.partials);
        k_adj_acc<<<1, kThreads, 0, st>>>(J.partials, kMassBlocks, 1, J.acc);
        int li = 0;
        for (long long sg = nseg - 1; sg >= 0 && e == cudaSuccess; --sg) {
            const long long start = sg * K;
            const long long len = (T - start) < K ? (T - start) : K;
            chk(cp(d.pop[d.cur], state(J.ckpt, sg)));
            chk(cp(state(J.seg, 0), d.pop[d.cur]));
            for (long long k = 1; k < len; ++k) {
                chk(step(d, kind, st, nullptr, nullptr));
                chk(cp(state(J.seg, k), d.pop[d.cur]));
            }
            for (long long k = len - 1; k >= 0; --k) {
                const S* x = reinterpret_cast<const S*>(state(J.seg, k));
                const S* lin = static_cast<const S*>(J.lam[li]);
                S* lout = static_cast<S*>(J.lam[1 - li]);
                adjoint_core(x, lin, std::false_type{});
                k_adj_pull<Q, S, SOLID, false><<<grid, kThreads, 0, st>>>(g, d.solid, dX, dJ, lin, P, lout, nullptr);
                li ^= 1;
            }
            chk(cudaGetLastError());
        }
        // initialisation: x(0) = equilibrium of the fields
        const S* x0 = reinterpret_cast<const S*>(state(J.ckpt, 0));
        adjoint_core(x0, static_cast<const S*>(J.lam[li]), std::true_type{});
        k_adj_pull<Q, S, SOLID, true><<<grid, kThreads, 0, st>>>(g, d.solid, dX, dJ, nullptr, P, nullptr, J.dfields);
        // leave the engine at x(T)
        d.cur = curT;
        chk(cp(d.pop[d.cur], J.fin));
        chk(cudaGetLastError());
        return e;
    }

    static cudaError_t adjoint(DevState& d, int kind, const tlbm_host::AdjJob& J, cudaStream_t st) {
        if constexpr (Fmt<Q, S>::PACKED) {  // 16-bit formats: no adjoint
            return cudaErrorNotSupported;
        } else {
            if (!d.mom) return cudaErrorInvalidValue;
            return d.solid ? adjoint_run<true>(d, kind, J, st) : adjoint_run<false>(d, kind, J, st);
        }
    }

    static cudaError_t bbuild(tlbm_host::BatchState& b, cudaStream_t st) { return batch_build<Q, S>(b, st); }
    static cudaError_t bstep(tlbm_host::BatchState& b, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1) {
        return batch_step<Q, S>(b, st, ev0, ev1);
    }

    static const tlbm_host::Ops* table() {
        static const tlbm_host::Ops o = {&step,     &init,         &fields,    &mass,   &get_box,
                                         &set_pops, &launches,     &aux_per_node, &has_fused, &bbuild,
                                         &bstep,    &adjoint};
        return &o;
    }
};

}  // namespace tlbm_dev

// the launch table of storage type S on lattice Q, as tlbm_host::NAME()
#define TLBM_DEFINE_OPS(NAME, S, Q)                                \
    namespace tlbm_host {                                          \
    const Ops* NAME() { return tlbm_dev::Impl<Q, S>::table(); }    \
    }
