// tlbm_adjoint.cuh -- discrete adjoint of the split time step (and of the
// equilibrium initialisation) of the ternary free-energy LB method
// (Semprebon, Krueger, Kusumaatmaja, arXiv:1511.02155), hand-written.
//
// Forward step at a fluid node r (pull form, x = stored post-collision state):
//   F_i(r)   = x_i(r - e_i), or x_{opp i}(r) when r - e_i is solid (bounce-back)
//   X(r)     = (rho, phi, psi) = sums of F; j = sum e_i f_i
//   X(s)     = wetting ghosts on solid nodes s from fluid axis neighbours
//              (mean of X(n) - G_X; diagonal-only: X(n) - sqrt 2 G_X)
//   grad, lap of X from the isotropic stencils over X (ghosts included)
//   eq(r)    = equilibria of (X, j, grad, lap) (Sec. Equations of Motion);
//              the rest population closes sum eq = X
//   x'_i(r)  = F_i + omega (eq_i - F_i)
// Its adjoint, given lambda = dL/dx' (stored in the population layout):
//   k_adj_node   per fluid node: the reverse of the node's equilibria and BGK
//                -> dL/dX(r) (local part), dL/dj, dL/dgrad, dL/dlap, dL/dkappa
//   k_adj_gather per node: transpose of the derivative stencils -> total dL/dX,
//                and on solid nodes the ghost's share of dL/dG_X
//   k_adj_pull   per fluid node: ghost transpose from solid neighbours, moment
//                transpose, the direct (1 - omega) lambda term, and the transpose
//                of the pull (a push) -> dL/dx of the previous state
// The initialisation x(0) = push(eq(fields)) has the same adjoint with omega = 1,
// no direct term and the pulled lambda; its last stage writes dL/dfields.
// Instantiated for FP64 and FP32 storage; the loss and the parameter gradients
// are always accumulated in FP64 (fixed-order block partials).
#pragma once

#include <type_traits>

#include "tlbm_kernels.cuh"

namespace tlbm_dev {

// ---------------------------------------------------------------- node adjoint

// Reverse of NodeEq::setup + NodeEq::eq + BGK at one node.  lam[s][i] = dL/dx'_i
// of set s (f, g, k).  om[s] = relaxation rates (1 for the initialisation).
// Adds to dX[3], dJ[3], dG[3][3] (dL/dgrad[X][a]), dLap[3], dKap[3].
template <int Q, typename T>
__host__ __device__ __forceinline__ void node_adjoint(const Phys<T>& P, const T X[3], const T j[3],
                                                      const T (&grad)[3][3], const T lap[3], const T (&lam)[3][Q],
                                                      const T om[3], T dX[3], T dJ[3], T (&dG)[3][3], T dLap[3],
                                                      T dKap[3]) {
    constexpr int D = Lat<Q>::D;
    const T rho = X[0], phi = X[1], psi = X[2];
    // ---- forward intermediates (the same expressions as NodeEq)
    const T inv = T(1) / rho;
    const T u[3] = {j[0] * inv, j[1] * inv, j[2] * inv};
    const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const T C[3] = {(rho + phi - psi) * T(0.5), (rho - phi - psi) * T(0.5), psi};
    const T lC[3] = {(lap[0] + lap[1] - lap[2]) * T(0.5), (lap[0] - lap[1] - lap[2]) * T(0.5), lap[2]};
    const T s3 = T(3) * P.a2;

    // ---- equilibria of i >= 1 and the rest closure
    T dbf = T(0), dbg = T(0), dbk = T(0), dGs[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    T du[3] = {T(0), T(0), T(0)};
    dX[0] += om[0] * lam[0][0];
    dX[1] += om[1] * lam[1][0];
    dX[2] += om[2] * lam[2][0];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const T af = om[0] * (lam[0][i] - lam[0][0]);
        const T ag = om[1] * (lam[1][i] - lam[1][0]);
        const T ak = om[2] * (lam[2][i] - lam[2][0]);
        const T w = T(Lat<Q>::w(i));
        T e = T(0);
        if (Lat<Q>::cx(i)) e += T(Lat<Q>::cx(i)) * u[0];
        if (Lat<Q>::cy(i)) e += T(Lat<Q>::cy(i)) * u[1];
        if (Lat<Q>::cz(i)) e += T(Lat<Q>::cz(i)) * u[2];
        const T poly = T(3) * e + T(4.5) * e * e;
        dbf += af * w;
        dbg += ag * w;
        dbk += ak * w;
        dX[0] += af * w * poly;
        dX[1] += ag * w * poly;
        dX[2] += ak * w * poly;
        const T de = w * (T(3) + T(9) * e) * (af * rho + ag * phi + ak * psi);
        if (Lat<Q>::cx(i)) du[0] += T(Lat<Q>::cx(i)) * de;
        if (Lat<Q>::cy(i)) du[1] += T(Lat<Q>::cy(i)) * de;
        if (Lat<Q>::cz(i)) du[2] += T(Lat<Q>::cz(i)) * de;
#pragma unroll
        for (int c = 0; c < 6; ++c)
            if (tens<Q>(i, c) != 0.0) dGs[c] += T(tens<Q>(i, c)) * af;
    }

    // ---- b_f, b_g, b_k
    const T dpb = T(3) * dbf;
    const T dLp = -s3 * dbf;
    const T duu = -T(1.5) * (rho * dbf + phi * dbg + psi * dbk);
    dX[0] += -T(1.5) * uu * dbf;
    dX[1] += -T(1.5) * uu * dbg;
    dX[2] += -T(1.5) * uu * dbk;
    const T dmphi = T(3) * P.gamma[0] * dbg;
    const T dmpsi = T(3) * P.gamma[1] * dbk;
    const T dmu[3] = {T(0.5) * dmphi - T(0.5) * dmpsi, -T(0.5) * dmphi - T(0.5) * dmpsi, dmpsi};

    // ---- chemical potentials and bulk pressure
    T dC[3], dlC[3];
    dX[0] += dpb * T(1.0 / 3.0);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const T c = C[m];
        const T b = c * (T(1) - c) * (T(1) - T(2) * c);
        const T bp = T(1) - T(6) * c + T(6) * c * c;
        const T p = c * c * (T(1) - c) * (T(1) - T(3) * c);
        const T pp = T(2) * c - T(12) * c * c + T(12) * c * c * c;
        dC[m] = dmu[m] * P.kappa[m] * bp + dpb * P.kappa[m] * T(0.5) * pp;
        dlC[m] = -dmu[m] * P.kappa[m] * P.a2;
        dKap[m] += dmu[m] * (b - P.a2 * lC[m]) + dpb * T(0.5) * p;
    }

    // ---- Laplacian part L = sum_ab X_a K_ab lap_b and gradient part Gs
    T dK[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T sa = T(0), sb = T(0);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            sa += P.K[a][b] * lap[b];
            sb += X[b] * P.K[b][a];
            dK[a][b] = dLp * X[a] * lap[b];
        }
        dX[a] += dLp * sa;
        dLap[a] += dLp * sb;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const int a = c < 3 ? c : c - 3;
        const int b = c < 3 ? c : (c - 3 + 1) % 3;
        if (a >= D || b >= D) continue;
        const T g = s3 * dGs[c];
#pragma unroll
        for (int x = 0; x < 3; ++x) {
            T kb = T(0), ka = T(0);
#pragma unroll
            for (int y = 0; y < 3; ++y) {
                kb += P.K[x][y] * grad[y][b];  // (K grad_b)_x
                ka += grad[y][a] * P.K[y][x];  // (grad_a^T K)_x
                dK[x][y] += g * grad[x][a] * grad[y][b];
            }
            dG[x][a] += g * kb;
            dG[x][b] += g * ka;
        }
    }
    // kappa through the mixing coefficients K(kappa)
    dKap[0] += T(0.25) * (dK[0][0] + dK[0][1] - dK[0][2] + dK[1][0] + dK[1][1] - dK[1][2] - dK[2][0] -
                          dK[2][1] + dK[2][2]);
    dKap[1] += T(0.25) * (dK[0][0] - dK[0][1] - dK[0][2] - dK[1][0] + dK[1][1] + dK[1][2] - dK[2][0] +
                          dK[2][1] + dK[2][2]);
    dKap[2] += dK[2][2];

    // ---- concentrations -> X, Laplacians of C -> Laplacians of X
    dX[0] += T(0.5) * (dC[0] + dC[1]);
    dX[1] += T(0.5) * (dC[0] - dC[1]);
    dX[2] += -T(0.5) * (dC[0] + dC[1]) + dC[2];
    dLap[0] += T(0.5) * (dlC[0] + dlC[1]);
    dLap[1] += T(0.5) * (dlC[0] - dlC[1]);
    dLap[2] += -T(0.5) * (dlC[0] + dlC[1]) + dlC[2];

    // ---- velocity u = j / rho
#pragma unroll
    for (int a = 0; a < 3; ++a) du[a] += T(2) * u[a] * duu;
    T udu = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dJ[a] += du[a] * inv;
        udu += du[a] * u[a];
    }
    dX[0] -= udu * inv;
}

// ------------------------------------------------------------------ helpers

// destination slot of the pulled population i of fluid node (x, y, z): the
// source node r - e_i, or the node itself (direction opp i) at a bounce-back
template <int Q, bool SOLID>
__device__ __forceinline__ void pull_slot(const Geom& g, const uint8_t* __restrict__ solid, int i, int x, int y,
                                          int z, int& xs, int& ys, int& zs, int& is) {
    xs = wrap(x - Lat<Q>::cx(i), g.nx);
    ys = wrap(y - Lat<Q>::cy(i), g.ny);
    zs = wrap(z - Lat<Q>::cz(i), g.nz);
    is = i;
    if (SOLID && solid[node(g, xs, ys, zs)]) {
        xs = x;
        ys = y;
        zs = z;
        is = opp<Q>(i);
    }
}

// ghost classification of solid node (x, y, z): fluid axis neighbours and fluid
// diagonal neighbours (the diagonal ones are used only when there is no axis one)
template <int Q>
__device__ __forceinline__ void ghost_counts(const Geom& g, const uint8_t* __restrict__ solid, int x, int y, int z,
                                             int& nax, int& ndg) {
    nax = 0;
    ndg = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const long long b = node(g, wrap(x + Lat<Q>::cx(i), g.nx), wrap(y + Lat<Q>::cy(i), g.ny),
                                 wrap(z + Lat<Q>::cz(i), g.nz));
        if (solid[b]) continue;
        if (i <= Lat<Q>::NAXIS) ++nax;
        else ++ndg;
    }
}

// ------------------------------------------------------------------ kernels

// Seed of the C_3 misfit L = sum_fluid (C_3(r) - target(r))^2 at state x:
// dL/dF^k_i(r) = 2 (psi(r) - target(r)), pushed into lam (the pull's transpose);
// solid nodes' own slots are zeroed.  Loss partials per block (fixed grid).
template <int Q, typename S, bool SOLID>
__global__ void __launch_bounds__(kThreads)
k_adj_seed(Geom g, const S* __restrict__ x, const uint8_t* __restrict__ solid, const double* __restrict__ target,
           S* __restrict__ lam, double* __restrict__ partials) {
    using T = typename Store<S>::T;
    double acc = 0.0;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
         r += (long long)gridDim.x * blockDim.x) {
        int xx, yy, zz;
        coords(g, r, xx, yy, zz);
        if (SOLID && solid[r]) {
#pragma unroll
            for (int s = 0; s < 3; ++s)
#pragma unroll
                for (int i = 0; i < Q; ++i) pst_raw<Q, S>(lam, g, s, i, xx, yy, zz, T(0));
            continue;
        }
        T psi = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) psi += pull_delta<Q, S, SOLID>(g, x, solid, 2, i, xx, yy, zz);
        const double d = (double)psi - target[r];
        acc += d * d;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            int xs, ys, zs, is;
            pull_slot<Q, SOLID>(g, solid, i, xx, yy, zz, xs, ys, zs, is);
            pst_raw<Q, S>(lam, g, 0, is, xs, ys, zs, T(0));
            pst_raw<Q, S>(lam, g, 1, is, xs, ys, zs, T(0));
            pst_raw<Q, S>(lam, g, 2, is, xs, ys, zs, T(2.0 * d));
        }
    }
    double z1 = 0.0, z2 = 0.0;
    block_sum3(acc, z1, z2);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Node adjoint at every fluid node.  STEP: populations pulled from x, lambda
// read at the node itself (x' of r is stored at r).  INIT: fields from mom,
// j = 0, omega = 1, lambda pulled (eq of r was pushed to the pull slots).
// Outputs node arrays dX[3][Np], dJ[3][Np], dG[9][Np] (dG[3X+a]), dLap[3][Np];
// kappa partials per block (fixed grid).
template <int Q, typename S, bool SOLID, bool INIT>
__global__ void __launch_bounds__(kThreads)
k_adj_node(Geom g, const S* __restrict__ x, const uint8_t* __restrict__ solid,
           const typename Store<S>::T* __restrict__ mom, const S* __restrict__ lam, Phys<typename Store<S>::T> P,
           typename Store<S>::T* __restrict__ dXo, typename Store<S>::T* __restrict__ dJo,
           typename Store<S>::T* __restrict__ dGo, typename Store<S>::T* __restrict__ dLo,
           double* __restrict__ partials) {
    using T = typename Store<S>::T;
    double k0 = 0.0, k1 = 0.0, k2 = 0.0;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
         r += (long long)gridDim.x * blockDim.x) {
        if (SOLID && solid[r]) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dXo[c * g.Np + r] = T(0);
                dJo[c * g.Np + r] = T(0);
                dLo[c * g.Np + r] = T(0);
            }
#pragma unroll
            for (int c = 0; c < 9; ++c) dGo[c * g.Np + r] = T(0);
            continue;
        }
        int xx, yy, zz;
        coords(g, r, xx, yy, zz);
        T X[3], j[3] = {T(0), T(0), T(0)}, om[3];
        T lm[3][Q];
        if (INIT) {
            X[0] = mom[r];
            X[1] = mom[g.Np + r];
            X[2] = mom[2 * g.Np + r];
            om[0] = om[1] = om[2] = T(1);
#pragma unroll
            for (int s = 0; s < 3; ++s)
#pragma unroll
                for (int i = 0; i < Q; ++i) lm[s][i] = pull_delta<Q, S, SOLID>(g, lam, solid, s, i, xx, yy, zz);
        } else {
            X[0] = X[1] = X[2] = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const T f = pull_delta<Q, S, SOLID>(g, x, solid, 0, i, xx, yy, zz);
                X[0] += f;
                if (Lat<Q>::cx(i)) j[0] += T(Lat<Q>::cx(i)) * f;
                if (Lat<Q>::cy(i)) j[1] += T(Lat<Q>::cy(i)) * f;
                if (Lat<Q>::cz(i)) j[2] += T(Lat<Q>::cz(i)) * f;
                X[1] += pull_delta<Q, S, SOLID>(g, x, solid, 1, i, xx, yy, zz);
                X[2] += pull_delta<Q, S, SOLID>(g, x, solid, 2, i, xx, yy, zz);
            }
            if (Fmt<Q, S>::OFFSET) X[0] += T(1);  // stored f deviations sum to rho - 1
            om[0] = P.omega[0];
            om[1] = P.omega[1];
            om[2] = P.omega[2];
            const unsigned char* b = reinterpret_cast<const unsigned char*>(lam) + node_off<Q, S>(g, xx, yy, zz);
#pragma unroll
            for (int s = 0; s < 3; ++s)
#pragma unroll
                for (int i = 0; i < Q; ++i) lm[s][i] = Fmt<Q, S>::ld_delta(b, s, i);
        }
        T grad[3][3], lap[3];
        derivs<Q, T>(g, mom, xx, yy, zz, r, grad, lap);
        T dX[3] = {T(0), T(0), T(0)}, dJ[3] = {T(0), T(0), T(0)}, dL[3] = {T(0), T(0), T(0)};
        T dG[3][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
        T dK[3] = {T(0), T(0), T(0)};
        node_adjoint<Q, T>(P, X, j, grad, lap, lm, om, dX, dJ, dG, dL, dK);
        k0 += (double)dK[0];
        k1 += (double)dK[1];
        k2 += (double)dK[2];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dXo[c * g.Np + r] = dX[c];
            dJo[c * g.Np + r] = dJ[c];
            dLo[c * g.Np + r] = dL[c];
#pragma unroll
            for (int a = 0; a < 3; ++a) dGo[(3 * c + a) * g.Np + r] = dG[c][a];
        }
    }
    block_sum3(k0, k1, k2);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = k0;
        partials[3 * blockIdx.x + 1] = k1;
        partials[3 * blockIdx.x + 2] = k2;
    }
}

// Transpose of the derivative stencils, at every node (in place on dX):
// dX(r) += sum_i [3 w_i e_i . dG(r - e_i) + 6 w_i dLap(r - e_i)] - 6 (1 - w_0) dLap(r).
// On solid nodes the total is the ghost's adjoint; its share of dL/dG_X
// (-1, or -sqrt 2 for diagonal-only ghosts) goes to per-block partials.
template <int Q, typename T, bool SOLID>
__global__ void __launch_bounds__(kThreads)
k_adj_gather(Geom g, const uint8_t* __restrict__ solid, T* __restrict__ dX, const T* __restrict__ dG,
             const T* __restrict__ dL, double* __restrict__ partials) {
    double p0 = 0.0, p1 = 0.0, p2 = 0.0;
    constexpr T wrest = T(1.0 - Lat<Q>::w(0));
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
         r += (long long)gridDim.x * blockDim.x) {
        int xx, yy, zz;
        coords(g, r, xx, yy, zz);
        T acc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c] = dX[c * g.Np + r] - T(6) * wrest * dL[c * g.Np + r];
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const long long b = node(g, wrap(xx - Lat<Q>::cx(i), g.nx), wrap(yy - Lat<Q>::cy(i), g.ny),
                                     wrap(zz - Lat<Q>::cz(i), g.nz));
            const T w = T(Lat<Q>::w(i));
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                T s = T(6) * dL[c * g.Np + b];
                if (Lat<Q>::cx(i)) s += T(3 * Lat<Q>::cx(i)) * dG[(3 * c + 0) * g.Np + b];
                if (Lat<Q>::cy(i)) s += T(3 * Lat<Q>::cy(i)) * dG[(3 * c + 1) * g.Np + b];
                if (Lat<Q>::cz(i)) s += T(3 * Lat<Q>::cz(i)) * dG[(3 * c + 2) * g.Np + b];
                acc[c] += w * s;
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) dX[c * g.Np + r] = acc[c];
        if (SOLID && solid[r]) {
            int nax, ndg;
            ghost_counts<Q>(g, solid, xx, yy, zz, nax, ndg);
            const double gc = nax > 0 ? 1.0 : (ndg > 0 ? 1.4142135623730951 : 0.0);
            p0 -= gc * (double)acc[0];
            p1 -= gc * (double)acc[1];
            p2 -= gc * (double)acc[2];
        }
    }
    block_sum3(p0, p1, p2);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = p0;
        partials[3 * blockIdx.x + 1] = p1;
        partials[3 * blockIdx.x + 2] = p2;
    }
}

// Last stage at every fluid node: the ghosts' transpose (solid neighbours s
// whose ghost used r pass dX(s)/n(s)), then
//   STEP: dL/dF_i = (1 - omega) lambda_i + [drho + e_i . dj | dphi | dpsi],
//         pushed to the pull slots of lam_out (solid nodes' own slots zeroed);
//   INIT: dL/dfields(r) = dX(r) into dfields[3][N] (solid nodes 0).
template <int Q, typename S, bool SOLID, bool INIT>
__global__ void __launch_bounds__(kThreads)
k_adj_pull(Geom g, const uint8_t* __restrict__ solid, const typename Store<S>::T* __restrict__ dXt,
           const typename Store<S>::T* __restrict__ dJ, const S* __restrict__ lam_in, Phys<typename Store<S>::T> P,
           S* __restrict__ lam_out, double* __restrict__ dfields) {
    using T = typename Store<S>::T;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
         r += (long long)gridDim.x * blockDim.x) {
        int xx, yy, zz;
        coords(g, r, xx, yy, zz);
        if (SOLID && solid[r]) {
            if (INIT) {
                dfields[r] = 0.0;
                dfields[g.N + r] = 0.0;
                dfields[2 * g.N + r] = 0.0;
            } else {
#pragma unroll
                for (int s = 0; s < 3; ++s)
#pragma unroll
                    for (int i = 0; i < Q; ++i) pst_raw<Q, S>(lam_out, g, s, i, xx, yy, zz, T(0));
            }
            continue;
        }
        T d[3] = {dXt[r], dXt[g.Np + r], dXt[2 * g.Np + r]};
        if (SOLID) {
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const int sx = wrap(xx + Lat<Q>::cx(i), g.nx), sy = wrap(yy + Lat<Q>::cy(i), g.ny),
                          sz = wrap(zz + Lat<Q>::cz(i), g.nz);
                const long long s = node(g, sx, sy, sz);
                if (!solid[s]) continue;
                int nax, ndg;
                ghost_counts<Q>(g, solid, sx, sy, sz, nax, ndg);
                const bool uses = (i <= Lat<Q>::NAXIS) ? (nax > 0) : (nax == 0 && ndg > 0);
                if (!uses) continue;
                const T inv = T(1) / T(i <= Lat<Q>::NAXIS ? nax : ndg);
#pragma unroll
                for (int c = 0; c < 3; ++c) d[c] += dXt[c * g.Np + s] * inv;
            }
        }
        if (INIT) {
            dfields[r] = (double)d[0];
            dfields[g.N + r] = (double)d[1];
            dfields[2 * g.N + r] = (double)d[2];
            continue;
        }
        const T dj[3] = {dJ[r], dJ[g.Np + r], dJ[2 * g.Np + r]};
        const unsigned char* lb = reinterpret_cast<const unsigned char*>(lam_in) + node_off<Q, S>(g, xx, yy, zz);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            T mf = d[0];
            if (Lat<Q>::cx(i)) mf += T(Lat<Q>::cx(i)) * dj[0];
            if (Lat<Q>::cy(i)) mf += T(Lat<Q>::cy(i)) * dj[1];
            if (Lat<Q>::cz(i)) mf += T(Lat<Q>::cz(i)) * dj[2];
            const T vf = (T(1) - P.omega[0]) * Fmt<Q, S>::ld_delta(lb, 0, i) + mf;
            const T vg = (T(1) - P.omega[1]) * Fmt<Q, S>::ld_delta(lb, 1, i) + d[1];
            const T vk = (T(1) - P.omega[2]) * Fmt<Q, S>::ld_delta(lb, 2, i) + d[2];
            int xs, ys, zs, is;
            pull_slot<Q, SOLID>(g, solid, i, xx, yy, zz, xs, ys, zs, is);
            pst_raw<Q, S>(lam_out, g, 0, is, xs, ys, zs, vf);
            pst_raw<Q, S>(lam_out, g, 1, is, xs, ys, zs, vg);
            pst_raw<Q, S>(lam_out, g, 2, is, xs, ys, zs, vk);
        }
    }
}

// acc[c] += sum over blocks k of partials[ncomp * k + c], in block order (one block)
static __global__ void k_adj_acc(const double* __restrict__ partials, int nblk, int ncomp, double* __restrict__ acc) {
    for (int c = 0; c < ncomp; ++c) {
        double a = 0.0, z1 = 0.0, z2 = 0.0;
        for (int k = threadIdx.x; k < nblk; k += blockDim.x) a += partials[ncomp * k + c];
        block_sum3(a, z1, z2);
        if (threadIdx.x == 0) acc[c] += a;
    }
}

}  // namespace tlbm_dev
