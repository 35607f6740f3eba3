// tlbm_guo.cuh -- the forcing coupling of the ternary free-energy LB step: the
// alternative that Sec. Equations of Motion mentions beside the pressure-tensor
// equilibrium, in which the thermodynamic terms enter the momentum equation as
// a body force with the source of Guo, Zheng and Shi (2002).
//
// The force is the divergence of the non-ideal part of the paper's pressure
// tensor,
//   F_a = -d_b Pi_ab,   Pi_ab = P_ab - rho c_s^2 delta_ab,
//   Pi_ab = alpha^2 G_ab + delta_ab [p_b - rho c_s^2 - alpha^2 (tr G / 2 + L)],
//   G_ab = sum_XY K_XY d_a X d_b Y,   L = sum_XY K_XY X lap Y,
// which in the continuum equals -(rho grad mu_rho + phi grad mu_phi + psi grad
// mu_psi) and on a periodic lattice sums to zero exactly (total momentum is
// conserved).  f relaxes to the ideal-gas equilibrium (pressure rho c_s^2) at
// the fluid velocity u = (j + F/2) / rho and receives
//   S_i = (1 - omega_f / 2) w_i [3 (e_i - u).F + 9 (e_i.u)(e_i.F)];
// g and k keep the equilibria of Sec. The Lattice Boltzmann Equation at the
// same u.  Periodic lattices only; every step is three launches:
//   k_moments       rho, phi, psi of the pulled populations   -> mom[3][Np]
//   k_guo_pressure  Pi (3 components on D2Q9, 6 on D3Q19) and
//                   mu_phi, mu_psi of every node               -> aux[NA][Np]
//   k_guo_collide   pull, F from Pi at the neighbours, collide with the
//                   source, store x*(r) in the other buffer
#pragma once

#include "tlbm_kernels.cuh"

namespace tlbm_dev {

// layout of the forcing coupling's node arrays aux[NA][Np]
template <int Q>
struct GuoAux {
    static constexpr int D = Lat<Q>::D;
    // Pi components: xx yy xy (D2Q9); xx yy zz xy yz zx (D3Q19)
    static constexpr int NPI = D == 2 ? 3 : 6;
    static constexpr int MU = NPI;  // mu_phi at MU, mu_psi at MU + 1
    static constexpr int NA = NPI + 2;
    // first and second axis of component c
    __host__ __device__ static constexpr int ca(int c) { return c < D ? c : c - D; }
    __host__ __device__ static constexpr int cb(int c) { return c < D ? c : (D == 2 ? 1 : (c - 2) % 3); }
    // component of the axis pair (a, b)
    __host__ __device__ static constexpr int comp(int a, int b) {
        return a == b ? a : (D == 2 ? 2 : (a + b == 1 ? 3 : (a + b == 3 ? 4 : 5)));
    }
};

// Pi and mu_phi, mu_psi of every node from the moment arrays (periodic).
template <int Q, typename T>
__global__ void __launch_bounds__(kThreads)
k_guo_pressure(Geom g, const T* __restrict__ mom, T* __restrict__ aux, Phys<T> P) {
    using A = GuoAux<Q>;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
         r += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(g, r, x, y, z);
        T grad[3][3], lap[3];
        derivs<Q, T>(g, mom, x, y, z, r, grad, lap);
        const T X[3] = {mom[r], mom[g.Np + r], mom[2 * g.Np + r]};
        // concentrations, chemical potentials and bulk pressure (Sec. Auxiliary
        // variables; p_b from the thermodynamic identity)
        const T C[3] = {(X[0] + X[1] - X[2]) * T(0.5), (X[0] - X[1] - X[2]) * T(0.5), X[2]};
        const T lC[3] = {(lap[0] + lap[1] - lap[2]) * T(0.5), (lap[0] - lap[1] - lap[2]) * T(0.5), lap[2]};
        T mu[3], pbx = T(0);  // pbx = p_b - rho c_s^2
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const T c = C[m], c1 = T(1) - c;
            mu[m] = P.kappa[m] * (c * c1 * (T(1) - T(2) * c) - P.a2 * lC[m]);
            pbx += P.kappa[m] * T(0.5) * c * c * c1 * (T(1) - T(3) * c);
        }
        // L = sum_XY K_XY X lap Y and G_ab = sum_XY K_XY d_a X d_b Y
        T Lp = T(0);
        T Kg[3][3];  // [X][b] = sum_Y K_XY d_b Y
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            T s = T(0);
#pragma unroll
            for (int b = 0; b < 3; ++b) s += P.K[a][b] * lap[b];
            Lp += X[a] * s;
#pragma unroll
            for (int b = 0; b < 3; ++b)
                Kg[a][b] = P.K[a][0] * grad[0][b] + P.K[a][1] * grad[1][b] + P.K[a][2] * grad[2][b];
        }
        T G[A::NPI];
        T trG = T(0);
#pragma unroll
        for (int c = 0; c < A::NPI; ++c) {
            const int a = A::ca(c), b = A::cb(c);
            G[c] = grad[0][a] * Kg[0][b] + grad[1][a] * Kg[1][b] + grad[2][a] * Kg[2][b];
            if (a == b) trG += G[c];
        }
        const T iso = pbx - P.a2 * (T(0.5) * trG + Lp);
#pragma unroll
        for (int c = 0; c < A::NPI; ++c)
            aux[c * g.Np + r] = P.a2 * G[c] + (A::ca(c) == A::cb(c) ? iso : T(0));
        aux[A::MU * g.Np + r] = (mu[0] - mu[1]) * T(0.5);
        aux[(A::MU + 1) * g.Np + r] = mu[2] - (mu[0] + mu[1]) * T(0.5);
    }
}

// F = -div Pi at (x, y, z): F_a = -3 sum_i w_i sum_b e_ib Pi_ab(r + e_i).
template <int Q, typename T>
__device__ __forceinline__ void guo_force(const Geom& g, const T* __restrict__ aux, int x, int y, int z,
                                          T (&F)[3]) {
    using A = GuoAux<Q>;
    F[0] = F[1] = F[2] = T(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const long long n = node(g, wrap(x + Lat<Q>::cx(i), g.nx), wrap(y + Lat<Q>::cy(i), g.ny),
                                 wrap(z + Lat<Q>::cz(i), g.nz));
        const int e[3] = {Lat<Q>::cx(i), Lat<Q>::cy(i), Lat<Q>::cz(i)};
        const T w = T(Lat<Q>::w(i));
#pragma unroll
        for (int a = 0; a < A::D; ++a) {
            T s = T(0);
#pragma unroll
            for (int b = 0; b < A::D; ++b)
                if (e[b]) s += T(e[b]) * aux[A::comp(a, b) * g.Np + n];
            F[a] -= w * s;
        }
    }
    F[0] *= T(3); F[1] *= T(3); F[2] *= T(3);
}

// Equilibria of direction i >= 1 under the forcing coupling, as deviations
// from Fmt::bias: f_eq = w_i rho (1 + 3 e.u + 4.5 (e.u)^2 - 1.5 u.u) (fb = rho,
// or rho - 1 where f is stored as f - w_i), g_eq = w_i (3 Gamma_phi mu_phi +
// phi (3 e.u + 4.5 (e.u)^2 - 1.5 u.u)), k_eq likewise with psi.
template <typename T>
struct GuoEq {
    T rho, phi, psi, fb, bg, bk, uu;
    __device__ __forceinline__ void eq(T w, T e, T& fe, T& ge, T& ke) const {
        const T q = T(3) * e + T(4.5) * e * e - T(1.5) * uu;
        fe = w * (fb + rho * q);
        ge = w * (bg + phi * q);
        ke = w * (bk + psi * q);
    }
};

// Collide and stream every node of a periodic lattice under the forcing
// coupling: pull, moments, F from Pi at the neighbours, u = (j + F/2) / rho,
// BGK towards the equilibria plus the Guo source (f only), store x*(r) in dst.
template <int Q, typename S>
__global__ void __launch_bounds__(kThreads)
k_guo_collide(Geom g, const S* __restrict__ src, S* __restrict__ dst,
              const typename Store<S>::T* __restrict__ aux, Phys<typename Store<S>::T> P) {
    using T = typename Store<S>::T;
    using A = GuoAux<Q>;
    constexpr bool OF = Fmt<Q, S>::OFFSET;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
         r += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(g, r, x, y, z);
        unsigned char* cb = reinterpret_cast<unsigned char*>(dst) + node_off<Q, S>(g, x, y, z);
        T f[Q], gg[Q], k[Q];  // f as stored (deviation where OF), g and k as they are
        T rd = T(0), j[3] = {T(0), T(0), T(0)}, phi = T(0), psi = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            f[i] = pull_delta<Q, S, false>(g, src, nullptr, 0, i, x, y, z);
            gg[i] = pull_delta<Q, S, false>(g, src, nullptr, 1, i, x, y, z);
            k[i] = pull_delta<Q, S, false>(g, src, nullptr, 2, i, x, y, z);
            rd += f[i];
            if (Lat<Q>::cx(i)) j[0] += T(Lat<Q>::cx(i)) * f[i];
            if (Lat<Q>::cy(i)) j[1] += T(Lat<Q>::cy(i)) * f[i];
            if (Lat<Q>::cz(i)) j[2] += T(Lat<Q>::cz(i)) * f[i];
            phi += gg[i];
            psi += k[i];
        }
        const T rho = OF ? T(1) + rd : rd;
        T F[3];
        guo_force<Q, T>(g, aux, x, y, z, F);
        const T inv = T(1) / rho;
        const T u[3] = {(j[0] + T(0.5) * F[0]) * inv, (j[1] + T(0.5) * F[1]) * inv,
                        (j[2] + T(0.5) * F[2]) * inv};
        GuoEq<T> E;
        E.rho = rho; E.phi = phi; E.psi = psi;
        E.fb = OF ? rd : rho;
        E.uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        E.bg = T(3) * P.gamma[0] * aux[A::MU * g.Np + r];
        E.bk = T(3) * P.gamma[1] * aux[(A::MU + 1) * g.Np + r];
        const T uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
        const T src_c = T(1) - T(0.5) * P.omega[0];
        T sf = T(0), sg = T(0), sk = T(0);  // sums of the moving equilibria (deviations)
        T qf = T(0), qg = T(0), qk = T(0);  // sums of the moving populations as stored
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            T e = T(0), eF = T(0);
            if (Lat<Q>::cx(i)) { e += T(Lat<Q>::cx(i)) * u[0]; eF += T(Lat<Q>::cx(i)) * F[0]; }
            if (Lat<Q>::cy(i)) { e += T(Lat<Q>::cy(i)) * u[1]; eF += T(Lat<Q>::cy(i)) * F[1]; }
            if (Lat<Q>::cz(i)) { e += T(Lat<Q>::cz(i)) * u[2]; eF += T(Lat<Q>::cz(i)) * F[2]; }
            const T w = T(Lat<Q>::w(i));
            T fe, ge, ke;
            E.eq(w, e, fe, ge, ke);
            sf += fe; sg += ge; sk += ke;
            const T Si = src_c * w * (T(3) * (eF - uF) + T(9) * e * eF);
            const T vf = f[i] + P.omega[0] * (fe - f[i]) + Si;
            const T vg = gg[i] + P.omega[1] * (ge - gg[i]);
            const T vk = k[i] + P.omega[2] * (ke - k[i]);
            Fmt<Q, S>::st_delta(cb, 0, i, vf);
            Fmt<Q, S>::st_delta(cb, 1, i, vg);
            Fmt<Q, S>::st_delta(cb, 2, i, vk);
            if (OF) {
                qf += Fmt<Q, S>::qdelta_d(i, vf);
                qg += Fmt<Q, S>::qdelta_d(i, vg);
                qk += Fmt<Q, S>::qdelta_d(i, vk);
            }
        }
        if (OF) {
            // the source sums to zero over i: the rest population is what keeps
            // the node's rho, phi, psi through the storage rounding
            Fmt<Q, S>::st_delta(cb, 0, 0, rd - qf);
            Fmt<Q, S>::st_delta(cb, 1, 0, phi - qg);
            Fmt<Q, S>::st_delta(cb, 2, 0, psi - qk);
        } else {
            const T S0 = src_c * T(Lat<Q>::w(0)) * (T(-3) * uF);
            Fmt<Q, S>::st_delta(cb, 0, 0, f[0] + P.omega[0] * ((rho - sf) - f[0]) + S0);
            Fmt<Q, S>::st_delta(cb, 1, 0, gg[0] + P.omega[1] * ((phi - sg) - gg[0]));
            Fmt<Q, S>::st_delta(cb, 2, 0, k[0] + P.omega[2] * ((psi - sk) - k[0]));
        }
    }
}

// Populations at the forcing coupling's equilibrium of the fields in mom (with
// mu_phi, mu_psi in aux; stored momentum rho u, u[3][N] or NULL for rest),
// scattered so that the pull yields x_i(r) = x_eq_i(r).  Periodic lattices.
template <int Q, typename S>
__global__ void __launch_bounds__(kThreads)
k_guo_init(Geom g, S* __restrict__ dst, const typename Store<S>::T* __restrict__ mom,
           const typename Store<S>::T* __restrict__ aux, const double* __restrict__ u,
           Phys<typename Store<S>::T> P) {
    using T = typename Store<S>::T;
    using A = GuoAux<Q>;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
         r += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(g, r, x, y, z);
        GuoEq<T> E;
        E.rho = mom[r]; E.phi = mom[g.Np + r]; E.psi = mom[2 * g.Np + r];
        E.fb = E.rho;
        const T v[3] = {u ? T(u[r]) : T(0), u ? T(u[g.N + r]) : T(0), u ? T(u[2 * g.N + r]) : T(0)};
        E.uu = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        E.bg = T(3) * P.gamma[0] * aux[A::MU * g.Np + r];
        E.bk = T(3) * P.gamma[1] * aux[(A::MU + 1) * g.Np + r];
        T eqv[3][Q];
        T sf = T(0), sg = T(0), sk = T(0);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            T e = T(0);
            if (Lat<Q>::cx(i)) e += T(Lat<Q>::cx(i)) * v[0];
            if (Lat<Q>::cy(i)) e += T(Lat<Q>::cy(i)) * v[1];
            if (Lat<Q>::cz(i)) e += T(Lat<Q>::cz(i)) * v[2];
            E.eq(T(Lat<Q>::w(i)), e, eqv[0][i], eqv[1][i], eqv[2][i]);
            sf += eqv[0][i]; sg += eqv[1][i]; sk += eqv[2][i];
        }
        eqv[0][0] = E.rho - sf; eqv[1][0] = E.phi - sg; eqv[2][0] = E.psi - sk;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int xs = wrap(x - Lat<Q>::cx(i), g.nx), ys = wrap(y - Lat<Q>::cy(i), g.ny),
                      zs = wrap(z - Lat<Q>::cz(i), g.nz);
#pragma unroll
            for (int s = 0; s < 3; ++s) pst<Q, S>(dst, g, s, i, xs, ys, zs, eqv[s][i]);
        }
    }
}

// Fluid velocity under the forcing coupling: u (holding j / rho) += F / (2 rho),
// with rho from mom and F from Pi in aux.  Periodic lattices.
template <int Q, typename T>
__global__ void __launch_bounds__(kThreads)
k_guo_velocity(Geom g, const T* __restrict__ mom, const T* __restrict__ aux, double* __restrict__ u) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
         r += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(g, r, x, y, z);
        T F[3];
        guo_force<Q, T>(g, aux, x, y, z, F);
        const double h = 0.5 / (double)mom[r];
#pragma unroll
        for (int a = 0; a < 3; ++a) u[a * g.N + r] += h * (double)F[a];
    }
}

}  // namespace tlbm_dev
