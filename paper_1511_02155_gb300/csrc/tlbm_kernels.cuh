// tlbm_kernels.cuh -- CUDA kernels of the ternary free-energy LB step
// (Semprebon, Krueger, Kusumaatmaja, arXiv:1511.02155) and the launch table
// that the C ABI dispatches through.
//
// Device state layout: one A-B pair of population buffers in the 32-node chunk
// layout of tlbm_lattice.cuh (Fmt), s = set (0 f, 1 g, 2 k), i = direction.
// The stored value at (i, r) is the POST-COLLISION population x*_i(r, t-1) of
// the previous step; the conventional population of the paper is recovered by
// the pull of Eq. latboltPropagation,
//   x_i(r, t) = x*_i(r - e_i, t-1)        if r - e_i is fluid,
//             = x*_{opp(i)}(r, t-1)        otherwise (halfway bounce-back).
// A step therefore reads with the pull, collides at r and writes x*(r, t) to
// the other buffer at r: every load of one warp is contiguous (shifted by at
// most one element) and every store is aligned.
#pragma once

#include "tlbm_internal.h"
#include "tlbm_lattice.cuh"

namespace tlbm_dev {

constexpr int kThreads = 256;

// physical parameters in the compute type
template <typename T>
inline Phys<T> to_phys(const tlbm_host::PhysD& p) {
    Phys<T> q;
    for (int m = 0; m < 3; ++m) {
        q.kappa[m] = T(p.kappa[m]);
        q.omega[m] = T(p.omega[m]);
        q.Gw[m] = T(p.Gw[m]);
        for (int n = 0; n < 3; ++n) q.K[m][n] = T(p.K[m][n]);
    }
    q.a2 = T(p.a2);
    q.gamma[0] = T(p.gamma[0]);
    q.gamma[1] = T(p.gamma[1]);
    return q;
}

constexpr int kMassBlocks = tlbm_host::kMassBlocks;  // fixed so reductions are repeatable

// ------------------------------------------------------------ small helpers

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum three doubles over the block in a fixed order; thread 0 gets the result.
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c) {
    __shared__ double sh[3][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
    if (lane == 0) { sh[0][wid] = a; sh[1][wid] = b; sh[2][wid] = c; }
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (wid == 0) {
        a = lane < nw ? sh[0][lane] : 0.0;
        b = lane < nw ? sh[1][lane] : 0.0;
        c = lane < nw ? sh[2][lane] : 0.0;
        a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
    }
    __syncthreads();
}

__device__ __forceinline__ void coords(const Geom& g, long long r, int& x, int& y, int& z) {
    x = (int)(r % g.nx);
    const long long t = r / g.nx;
    y = (int)(t % g.ny);
    z = (int)(t / g.ny);
}

// Pulled (conventional) population i of set s at fluid node r = (x, y, z).
template <int Q, typename S, bool SOLID>
__device__ __forceinline__ typename Store<S>::T pull(const Geom& g, const S* __restrict__ src,
                                                      const uint8_t* __restrict__ solid, int s,
                                                      int i, int x, int y, int z, long long r) {
    const int xs = wrap(x - Lat<Q>::cx(i), g.nx), ys = wrap(y - Lat<Q>::cy(i), g.ny),
              zs = wrap(z - Lat<Q>::cz(i), g.nz);
    if (SOLID && solid[node(g, xs, ys, zs)]) return pld<Q, S>(src, g, s, opp<Q>(i), x, y, z);
    return pld<Q, S>(src, g, s, i, xs, ys, zs);
}

// The same population as stored: its deviation from Fmt::bias (f_i - w_i in the
// 16-bit formats, the value itself otherwise).
template <int Q, typename S, bool SOLID>
__device__ __forceinline__ typename Store<S>::T pull_delta(const Geom& g, const S* __restrict__ src,
                                                            const uint8_t* __restrict__ solid, int s,
                                                            int i, int x, int y, int z) {
    const int xs = wrap(x - Lat<Q>::cx(i), g.nx), ys = wrap(y - Lat<Q>::cy(i), g.ny),
              zs = wrap(z - Lat<Q>::cz(i), g.nz);
    const unsigned char* b = reinterpret_cast<const unsigned char*>(src);
    if (SOLID && solid[node(g, xs, ys, zs)]) return Fmt<Q, S>::ld_delta(b + node_off<Q, S>(g, x, y, z), s, opp<Q>(i));
    return Fmt<Q, S>::ld_delta(b + node_off<Q, S>(g, xs, ys, zs), s, i);
}

// rho of a node from the sum rd of its stored f deviations (16-bit formats keep
// f - w, whose sum is rho - 1)
template <int Q, typename S>
__device__ __forceinline__ double rho_total(typename Store<S>::T rd) {
    return Fmt<Q, S>::OFFSET ? 1.0 + (double)rd : (double)rd;
}

// ------------------------------------------------- moments (+ mass partials)

// Moments rho, phi, psi of every fluid node from the pulled populations; writes
// them to mom[3][Np] when WRITE, and the block's FP64 totals to partials[blk].
// Grid-stride over a fixed grid of kMassBlocks blocks.
template <int Q, typename S, bool SOLID, bool WRITE>
__global__ void __launch_bounds__(kThreads)
k_moments(Geom g, const S* __restrict__ src, const uint8_t* __restrict__ solid,
          typename Store<S>::T* __restrict__ mom, double* __restrict__ partials) {
    using T = typename Store<S>::T;
    double sr = 0.0, sp = 0.0, ss = 0.0;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
         r += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(g, r, x, y, z);
        T rd = T(0), phi = T(0), psi = T(0);
        if (!(SOLID && solid[r])) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                rd += pull_delta<Q, S, SOLID>(g, src, solid, 0, i, x, y, z);
                phi += pull_delta<Q, S, SOLID>(g, src, solid, 1, i, x, y, z);
                psi += pull_delta<Q, S, SOLID>(g, src, solid, 2, i, x, y, z);
            }
            sr += rho_total<Q, S>(rd); sp += (double)phi; ss += (double)psi;
        }
        const T rho = (SOLID && solid[r]) ? T(0) : T(rho_total<Q, S>(rd));
        if (WRITE) {
            mom[r] = rho;
            mom[g.Np + r] = phi;
            mom[2 * g.Np + r] = psi;
        }
    }
    block_sum3(sr, sp, ss);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = sr;
        partials[3 * blockIdx.x + 1] = sp;
        partials[3 * blockIdx.x + 2] = ss;
    }
}

// Sum the block partials in a fixed order; raise the flag if not finite.
static __global__ void k_mass_final(const double* __restrict__ partials, int nblk, double* __restrict__ out,
                             int* __restrict__ flag) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int k = threadIdx.x; k < nblk; k += blockDim.x) {
        a += partials[3 * k]; b += partials[3 * k + 1]; c += partials[3 * k + 2];
    }
    block_sum3(a, b, c);
    if (threadIdx.x == 0) {
        out[0] = a; out[1] = b; out[2] = c;
        if (!(isfinite(a) && isfinite(b) && isfinite(c))) *flag = 1;
    }
}

// ------------------------------------------------------------ wetting ghosts

// Solid nodes next to fluid take X(s) = mean over fluid axis neighbours n of
// X(n) - G_X; with only diagonal fluid neighbours, the mean of X(n) - sqrt(2) G_X.
// G_X is the wall-normal gradient that the wetting condition prescribes.
template <int Q, typename T>
__global__ void __launch_bounds__(kThreads)
k_ghosts(Geom g, const uint8_t* __restrict__ solid, T* __restrict__ mom, Phys<T> P) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
         r += (long long)gridDim.x * blockDim.x) {
        if (!solid[r]) continue;
        int x, y, z;
        coords(g, r, x, y, z);
        T acc[3] = {T(0), T(0), T(0)};
        int n = 0;
#pragma unroll
        for (int i = 1; i <= Lat<Q>::NAXIS; ++i) {
            const long long b = node(g, wrap(x + Lat<Q>::cx(i), g.nx), wrap(y + Lat<Q>::cy(i), g.ny),
                                     wrap(z + Lat<Q>::cz(i), g.nz));
            if (solid[b]) continue;
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[c] += mom[c * g.Np + b] - P.Gw[c];
            ++n;
        }
        if (n == 0) {
            const T r2 = T(1.4142135623730951);
#pragma unroll
            for (int i = Lat<Q>::NAXIS + 1; i < Q; ++i) {
                const long long b = node(g, wrap(x + Lat<Q>::cx(i), g.nx),
                                         wrap(y + Lat<Q>::cy(i), g.ny), wrap(z + Lat<Q>::cz(i), g.nz));
                if (solid[b]) continue;
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[c] += mom[c * g.Np + b] - r2 * P.Gw[c];
                ++n;
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) mom[c * g.Np + r] = n > 0 ? acc[c] / T(n) : T(0);
    }
}

// ---------------------------------------------------------- derivatives

// Isotropic gradient and Laplacian of the three moment fields at (x, y, z)
// from mom[3][Np]: d_a X = 3 sum_i w_i e_ia X(r+e_i), lap X = 6 sum_i w_i (X(r+e_i) - X(r)).
template <int Q, typename T>
__device__ __forceinline__ void derivs(const Geom& g, const T* __restrict__ mom, int x, int y,
                                       int z, long long r, T (&grad)[3][3], T (&lap)[3]) {
    T X0[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        X0[c] = mom[c * g.Np + r];
        lap[c] = T(0);
        grad[c][0] = grad[c][1] = grad[c][2] = T(0);
    }
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const long long b = node(g, wrap(x + Lat<Q>::cx(i), g.nx), wrap(y + Lat<Q>::cy(i), g.ny),
                                 wrap(z + Lat<Q>::cz(i), g.nz));
        const T w = T(Lat<Q>::w(i));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T v = mom[c * g.Np + b];
            if (Lat<Q>::cx(i)) grad[c][0] += T(Lat<Q>::cx(i)) * w * v;
            if (Lat<Q>::cy(i)) grad[c][1] += T(Lat<Q>::cy(i)) * w * v;
            if (Lat<Q>::cz(i)) grad[c][2] += T(Lat<Q>::cz(i)) * w * v;
            lap[c] += w * (v - X0[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        grad[c][0] *= T(3); grad[c][1] *= T(3); grad[c][2] *= T(3);
        lap[c] *= T(6);
    }
}

// ------------------------------------------------------- split collide step

// Collide and stream every fluid node: pull populations, moments, derivatives
// of the moment arrays (ghosts already on solid nodes), equilibria, BGK, store
// x* at r in dst.  Solid nodes store zeros.
template <int Q, typename S, bool SOLID>
__global__ void __launch_bounds__(kThreads)
k_collide_split(Geom g, const S* __restrict__ src, S* __restrict__ dst,
                const uint8_t* __restrict__ solid, const typename Store<S>::T* __restrict__ mom,
                Phys<typename Store<S>::T> P) {
    using T = typename Store<S>::T;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
         r += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(g, r, x, y, z);
        unsigned char* cb = reinterpret_cast<unsigned char*>(dst) + node_off<Q, S>(g, x, y, z);
        if (SOLID && solid[r]) {
#pragma unroll
            for (int s = 0; s < 3; ++s)
#pragma unroll
                for (int i = 0; i < Q; ++i) Fmt<Q, S>::st(cb, s, i, T(Fmt<Q, S>::bias(s, i)));
            continue;
        }
        T f[Q], gg[Q], k[Q];
        T rd = T(0), jx = T(0), jy = T(0), jz = T(0), phi = T(0), psi = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T fd = pull_delta<Q, S, SOLID>(g, src, solid, 0, i, x, y, z);
            f[i] = fd + T(Fmt<Q, S>::bias(0, i));
            gg[i] = pull_delta<Q, S, SOLID>(g, src, solid, 1, i, x, y, z);
            k[i] = pull_delta<Q, S, SOLID>(g, src, solid, 2, i, x, y, z);
            rd += fd;
            if (Lat<Q>::cx(i)) jx += T(Lat<Q>::cx(i)) * fd;
            if (Lat<Q>::cy(i)) jy += T(Lat<Q>::cy(i)) * fd;
            if (Lat<Q>::cz(i)) jz += T(Lat<Q>::cz(i)) * fd;
            phi += gg[i];
            psi += k[i];
        }
        const T rho = Fmt<Q, S>::OFFSET ? T(1) + rd : rd;
        T grad[3][3], lap[3];
        derivs<Q, T>(g, mom, x, y, z, r, grad, lap);
        NodeEq<Q, T> E;
        E.setup(P, rho, jx, jy, jz, phi, psi, grad, lap);
        T sf = T(0), sg = T(0), sk = T(0);  // sums of the moving equilibria
        T qf = T(0), qg = T(0), qk = T(0);  // sums of the moving populations as stored
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            T fe, ge, ke;
            E.eq(i, fe, ge, ke);
            sf += fe; sg += ge; sk += ke;
            const T vf = f[i] + P.omega[0] * (fe - f[i]);
            const T vg = gg[i] + P.omega[1] * (ge - gg[i]);
            const T vk = k[i] + P.omega[2] * (ke - k[i]);
            Fmt<Q, S>::st(cb, 0, i, vf);
            Fmt<Q, S>::st(cb, 1, i, vg);
            Fmt<Q, S>::st(cb, 2, i, vk);
            if (Fmt<Q, S>::OFFSET) {
                qf += Fmt<Q, S>::qdelta(0, i, vf);
                qg += Fmt<Q, S>::qdelta(1, i, vg);
                qk += Fmt<Q, S>::qdelta(2, i, vk);
            }
        }
        if (Fmt<Q, S>::OFFSET) {
            // rest = moment - moving populations as stored (deviations for f):
            // every node keeps its rho, phi, psi through the storage rounding
            Fmt<Q, S>::st_delta(cb, 0, 0, rd - qf);
            Fmt<Q, S>::st_delta(cb, 1, 0, phi - qg);
            Fmt<Q, S>::st_delta(cb, 2, 0, psi - qk);
        } else {
            Fmt<Q, S>::st(cb, 0, 0, f[0] + P.omega[0] * ((rho - sf) - f[0]));
            Fmt<Q, S>::st(cb, 1, 0, gg[0] + P.omega[1] * ((phi - sg) - gg[0]));
            Fmt<Q, S>::st(cb, 2, 0, k[0] + P.omega[2] * ((psi - sk) - k[0]));
        }
    }
}

// ------------------------------------------------------------ initialisation

// Moment arrays from host-supplied double fields (solid nodes zero).
template <typename T>
__global__ void k_fields_to_mom(Geom g, const double* __restrict__ rho, const double* __restrict__ phi,
                                const double* __restrict__ psi, const uint8_t* __restrict__ solid,
                                T* __restrict__ mom) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
         r += (long long)gridDim.x * blockDim.x) {
        const bool s = solid && solid[r];
        mom[r] = s ? T(0) : T(rho[r]);
        mom[g.Np + r] = s ? T(0) : T(phi[r]);
        mom[2 * g.Np + r] = s ? T(0) : T(psi[r]);
    }
}

// Equilibria of the fields (moments and ghosts in mom, velocity u[3][N] or NULL),
// scattered into storage so that the pull yields f_i(r) = f_eq_i(r).
template <int Q, typename S, bool SOLID>
__global__ void __launch_bounds__(kThreads)
k_init_eq(Geom g, S* __restrict__ dst, const uint8_t* __restrict__ solid,
          const typename Store<S>::T* __restrict__ mom, const double* __restrict__ u,
          Phys<typename Store<S>::T> P) {
    using T = typename Store<S>::T;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
         r += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(g, r, x, y, z);
        if (SOLID && solid[r]) {
#pragma unroll
            for (int s = 0; s < 3; ++s)
#pragma unroll
                for (int i = 0; i < Q; ++i) pst<Q, S>(dst, g, s, i, x, y, z, T(Fmt<Q, S>::bias(s, i)));
            continue;
        }
        const T rho = mom[r], phi = mom[g.Np + r], psi = mom[2 * g.Np + r];
        const T jx = u ? rho * T(u[r]) : T(0);
        const T jy = u ? rho * T(u[g.N + r]) : T(0);
        const T jz = u ? rho * T(u[2 * g.N + r]) : T(0);
        T grad[3][3], lap[3];
        derivs<Q, T>(g, mom, x, y, z, r, grad, lap);
        NodeEq<Q, T> E;
        E.setup(P, rho, jx, jy, jz, phi, psi, grad, lap);
        T eqv[3][Q];
        T sf = T(0), sg = T(0), sk = T(0);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            E.eq(i, eqv[0][i], eqv[1][i], eqv[2][i]);
            sf += eqv[0][i]; sg += eqv[1][i]; sk += eqv[2][i];
        }
        eqv[0][0] = rho - sf; eqv[1][0] = phi - sg; eqv[2][0] = psi - sk;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int xs = wrap(x - Lat<Q>::cx(i), g.nx), ys = wrap(y - Lat<Q>::cy(i), g.ny),
                      zs = wrap(z - Lat<Q>::cz(i), g.nz);
            const bool bounce = SOLID && solid[node(g, xs, ys, zs)];
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                if (bounce) pst<Q, S>(dst, g, s, opp<Q>(i), x, y, z, eqv[s][i]);
                else pst<Q, S>(dst, g, s, i, xs, ys, zs, eqv[s][i]);
            }
        }
    }
}

// -------------------------------------------------------------- read-back

// Macroscopic fields C1, C2, C3, rho, u[3] (doubles, any pointer may be NULL).
template <int Q, typename S, bool SOLID>
__global__ void __launch_bounds__(kThreads)
k_fields(Geom g, const S* __restrict__ src, const uint8_t* __restrict__ solid, double* __restrict__ C1,
         double* __restrict__ C2, double* __restrict__ C3, double* __restrict__ rho_out,
         double* __restrict__ u) {
    using T = typename Store<S>::T;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
         r += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(g, r, x, y, z);
        T rd = T(0), jx = T(0), jy = T(0), jz = T(0), phi = T(0), psi = T(0);
        const bool s = SOLID && solid[r];
        if (!s) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const T fd = pull_delta<Q, S, SOLID>(g, src, solid, 0, i, x, y, z);
                rd += fd;
                if (Lat<Q>::cx(i)) jx += T(Lat<Q>::cx(i)) * fd;
                if (Lat<Q>::cy(i)) jy += T(Lat<Q>::cy(i)) * fd;
                if (Lat<Q>::cz(i)) jz += T(Lat<Q>::cz(i)) * fd;
                phi += pull_delta<Q, S, SOLID>(g, src, solid, 1, i, x, y, z);
                psi += pull_delta<Q, S, SOLID>(g, src, solid, 2, i, x, y, z);
            }
        }
        const double dr = s ? 0.0 : rho_total<Q, S>(rd), dp = (double)phi, ds = (double)psi;
        if (C1) C1[r] = s ? 0.0 : 0.5 * (dr + dp - ds);
        if (C2) C2[r] = s ? 0.0 : 0.5 * (dr - dp - ds);
        if (C3) C3[r] = s ? 0.0 : ds;
        if (rho_out) rho_out[r] = s ? 0.0 : dr;
        if (u) {
            u[r] = s ? 0.0 : (double)jx / dr;
            u[g.N + r] = s ? 0.0 : (double)jy / dr;
            u[2 * g.N + r] = s ? 0.0 : (double)jz / dr;
        }
    }
}

// Conventional populations of a box (coordinates wrap) as doubles [s][i][b].
template <int Q, typename S, bool SOLID>
__global__ void __launch_bounds__(kThreads)
k_get_box(Geom g, const S* __restrict__ src, const uint8_t* __restrict__ solid, int x0, int y0,
          int z0, int bx, int by, int bz, double* __restrict__ out) {
    const long long nb = (long long)bx * by * bz;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
         b += (long long)gridDim.x * blockDim.x) {
        const int lx = (int)(b % bx);
        const int ly = (int)((b / bx) % by);
        const int lz = (int)(b / ((long long)bx * by));
        const int x = ((x0 + lx) % g.nx + g.nx) % g.nx;
        const int y = ((y0 + ly) % g.ny + g.ny) % g.ny;
        const int z = ((z0 + lz) % g.nz + g.nz) % g.nz;
        const long long r = node(g, x, y, z);
        const bool s = SOLID && solid[r];
#pragma unroll
        for (int set = 0; set < 3; ++set)
#pragma unroll
            for (int i = 0; i < Q; ++i)
                out[(long long)(set * Q + i) * nb + b] =
                    s ? 0.0 : (double)pull<Q, S, SOLID>(g, src, solid, set, i, x, y, z, r);
    }
}

// Storage from conventional double populations in[3][Q][N] (inverse of the pull).
template <int Q, typename S, bool SOLID>
__global__ void __launch_bounds__(kThreads)
k_set_pops(Geom g, const double* __restrict__ in, const uint8_t* __restrict__ solid, S* __restrict__ dst) {
    using T = typename Store<S>::T;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
         r += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(g, r, x, y, z);
        const bool s = SOLID && solid[r];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            // x*_i(r) = f_i(r + e_i) if that node is fluid, else f_opp(i)(r)
            const long long q = node(g, wrap(x + Lat<Q>::cx(i), g.nx), wrap(y + Lat<Q>::cy(i), g.ny),
                                     wrap(z + Lat<Q>::cz(i), g.nz));
            const bool bounce = SOLID && solid[q];
#pragma unroll
            for (int set = 0; set < 3; ++set) {
                const double v = bounce ? in[(long long)(set * Q + opp<Q>(i)) * g.N + r]
                                        : in[(long long)(set * Q + i) * g.N + q];
                pst<Q, S>(dst, g, set, i, x, y, z, s ? T(Fmt<Q, S>::bias(set, i)) : T(v));
            }
        }
    }
}

}  // namespace tlbm_dev
