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
// same u.  Periodic lattices only.  The marching kernel k_guo_fused (below)
// does a step in one launch; the split step is three launches:
//   k_moments       rho, phi, psi of the pulled populations   -> mom[3][Np]
//   k_guo_pressure  Pi (3 components on D2Q9, 6 on D3Q19) and
//                   mu_phi, mu_psi of every node               -> aux[NA][Np]
//   k_guo_collide   pull, F from Pi at the neighbours, collide with the
//                   source, store x*(r) in the other buffer
#pragma once

#include "tlbm_fused.cuh"
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

// Pi (GuoAux components) and mu_phi, mu_psi of one node from its fields X =
// (rho, phi, psi), their gradients grad[X][axis] and Laplacians lap[X].
template <int Q, typename T>
__device__ __forceinline__ void guo_node(const Phys<T>& P, const T (&X)[3], const T (&grad)[3][3],
                                         const T (&lap)[3], T (&pi)[GuoAux<Q>::NPI], T& mu_phi, T& mu_psi) {
    using A = GuoAux<Q>;
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
    for (int c = 0; c < A::NPI; ++c) pi[c] = P.a2 * G[c] + (A::ca(c) == A::cb(c) ? iso : T(0));
    mu_phi = (mu[0] - mu[1]) * T(0.5);
    mu_psi = mu[2] - (mu[0] + mu[1]) * T(0.5);
}

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
        T pi[A::NPI], mp, ms;
        guo_node<Q, T>(P, X, grad, lap, pi, mp, ms);
#pragma unroll
        for (int c = 0; c < A::NPI; ++c) aux[c * g.Np + r] = pi[c];
        aux[A::MU * g.Np + r] = mp;
        aux[(A::MU + 1) * g.Np + r] = ms;
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

// BGK of one node under the forcing coupling towards the equilibria plus the
// Guo source (f only), stored at node pointer cb.  f, gg, k: the pulled
// populations as stored (f as deviations where Fmt::OFFSET); rd their summed f
// (rho - 1 where OFFSET, else rho); j the momentum, F the force (lattice axes);
// bg, bk = 3 Gamma mu_phi, 3 Gamma mu_psi.
template <int Q, typename S>
__device__ __forceinline__ void guo_collide_node(unsigned char* cb, const typename Store<S>::T (&f)[Q],
                                                 const typename Store<S>::T (&gg)[Q],
                                                 const typename Store<S>::T (&k)[Q], typename Store<S>::T rd,
                                                 const typename Store<S>::T (&j)[3], typename Store<S>::T phi,
                                                 typename Store<S>::T psi, const typename Store<S>::T (&F)[3],
                                                 typename Store<S>::T bg, typename Store<S>::T bk,
                                                 const Phys<typename Store<S>::T>& P) {
    using T = typename Store<S>::T;
    constexpr bool OF = Fmt<Q, S>::OFFSET;
    const T rho = OF ? T(1) + rd : rd;
    const T inv = T(1) / rho;
    const T u[3] = {(j[0] + T(0.5) * F[0]) * inv, (j[1] + T(0.5) * F[1]) * inv, (j[2] + T(0.5) * F[2]) * inv};
    GuoEq<T> E;
    E.rho = rho; E.phi = phi; E.psi = psi;
    E.fb = OF ? rd : rho;
    E.uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    E.bg = bg;
    E.bk = bk;
    const T uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    const T src_c = T(1) - T(0.5) * P.omega[0];
    T sf = T(0), sg = T(0), sk = T(0);  // sums of the moving equilibria (deviations)
    T qf = T(0), qg = T(0), qk = T(0);  // sums of the moving populations as stored
    // opposite directions in pairs, so that the paired lane words are stored whole
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int o = opp<Q>(i);
        if (o < i) continue;
        T vf[2], vg[2], vk[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int d = h ? o : i;
            T e = T(0), eF = T(0);
            if (Lat<Q>::cx(d)) { e += T(Lat<Q>::cx(d)) * u[0]; eF += T(Lat<Q>::cx(d)) * F[0]; }
            if (Lat<Q>::cy(d)) { e += T(Lat<Q>::cy(d)) * u[1]; eF += T(Lat<Q>::cy(d)) * F[1]; }
            if (Lat<Q>::cz(d)) { e += T(Lat<Q>::cz(d)) * u[2]; eF += T(Lat<Q>::cz(d)) * F[2]; }
            const T w = T(Lat<Q>::w(d));
            T fe, ge, ke;
            E.eq(w, e, fe, ge, ke);
            sf += fe; sg += ge; sk += ke;
            const T Si = src_c * w * (T(3) * (eF - uF) + T(9) * e * eF);
            vf[h] = f[d] + P.omega[0] * (fe - f[d]) + Si;
            vg[h] = gg[d] + P.omega[1] * (ge - gg[d]);
            vk[h] = k[d] + P.omega[2] * (ke - k[d]);
            if (OF) {
                qf += Fmt<Q, S>::qdelta_d(d, vf[h]);
                qg += Fmt<Q, S>::qdelta_d(d, vg[h]);
                qk += Fmt<Q, S>::qdelta_d(d, vk[h]);
            }
        }
        Fmt<Q, S>::template st_fg<false>(cb, i, vf[0], vg[0]);
        Fmt<Q, S>::template st_fg<false>(cb, o, vf[1], vg[1]);
        Fmt<Q, S>::template st_kk<false>(cb, i, vk[0], vk[1]);
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

// Collide and stream every node of a periodic lattice under the forcing
// coupling: pull, moments, F from Pi at the neighbours, guo_collide_node.
template <int Q, typename S>
__global__ void __launch_bounds__(kThreads)
k_guo_collide(Geom g, const S* __restrict__ src, S* __restrict__ dst,
              const typename Store<S>::T* __restrict__ aux, Phys<typename Store<S>::T> P) {
    using T = typename Store<S>::T;
    using A = GuoAux<Q>;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
         r += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(g, r, x, y, z);
        unsigned char* cb = reinterpret_cast<unsigned char*>(dst) + node_off<Q, S>(g, x, y, z);
        T f[Q], gg[Q], k[Q];  // f as stored (deviation where OFFSET), g and k as they are
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
        T F[3];
        guo_force<Q, T>(g, aux, x, y, z, F);
        guo_collide_node<Q, S>(cb, f, gg, k, rd, j, phi, psi, F, T(3) * P.gamma[0] * aux[A::MU * g.Np + r],
                               T(3) * P.gamma[1] * aux[(A::MU + 1) * g.Np + r], P);
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

// ------------------------------------------------ one marching kernel per step

// The forcing coupling's step as one kernel (periodic lattices), on the
// marching scheme of k_fused: a block owns a TX x TY column tile and marches a
// chunk of planes.  F at r needs Pi at r's neighbours, and Pi the derivatives
// of the moments, so the block keeps a two-node halo of moments and a one-node
// halo of Pi and works two planes ahead:
//   M(m+2): moments of plane m+2 over tile + two-node halo   -> moment ring
//   barrier
//   P(m+1): Pi of plane m+1 over tile + one-node halo          -> Pi ring
//   barrier
//   C(m):   mu_phi, mu_psi from the moment ring's Laplacians, F from the Pi
//           ring, pull, guo_collide_node, store x*(r).
// Ring slots: moments five (a fast warp writes plane m+2 while a slow one still
// reads planes m-2..m in C(m-1)); Pi three (P(m+1) starts after the barrier
// that every warp reaches only once its C(m-1), the last reader of plane
// m-2, is done); momentum four.
template <int Q, typename S, int TX, int TY>
__device__ __forceinline__ void guo_body(const MGeom& g, const S* __restrict__ src, S* __restrict__ dst,
                                         const Phys<typename Store<S>::T>& P, double* __restrict__ partials,
                                         const int bid) {
    using T = typename Store<S>::T;
    using A = Axes<Q>;
    using GA = GuoAux<Q>;
    constexpr int D = Lat<Q>::D;
    constexpr int H = 2;                  // moment halo along a
    constexpr int HB = (D == 3) ? 2 : 0;  // moment halo along b
    constexpr int HW = TX + 2 * H;
    constexpr int HH = TY + 2 * HB;
    constexpr int HN = HW * HH;
    constexpr int NT = TX * TY;
    constexpr int KS = (HN + NT - 1) / NT;  // moment-region nodes per thread
    constexpr int PB = (D == 3) ? 1 : 0;    // Pi halo along b (one node along a)
    constexpr int PW = TX + 2;
    constexpr int PN = PW * (TY + 2 * PB);
    constexpr int KP = (PN + NT - 1) / NT;  // Pi-region nodes per thread
    constexpr int NPI = GA::NPI;
    static_assert(D == 3 || TY == 1, "2-D tiles are one row");
    static_assert(KS <= 3 && KP <= 2, "region nodes per thread");

    __shared__ T sm[5][3][HN];    // rho, phi, psi over tile + two-node halo
    __shared__ T sp[3][NPI][PN];  // Pi over tile + one-node halo
    __shared__ T sj[4][4][NT];    // j (marching axes) and summed f of the tile

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int tileA = bid % g.tilesA;
    const int rest = bid / g.tilesA;
    const int tileB = rest % g.tilesB;
    const int chunk = rest / g.tilesB;
    const int A0 = tileA * TX, B0 = tileB * TY;
    const int M0 = (int)((long long)chunk * g.NM / g.NC);
    const int M1 = (int)((long long)(chunk + 1) * g.NM / g.NC);
    const bool active = (A0 + tx < g.NA) && (B0 + ty < g.NB);

    // moment-region nodes of this thread: pull-source byte offsets along a, rows along b
    int xc[KS][3], yb[KS][3];
#pragma unroll
    for (int k = 0; k < KS; ++k) {
        const int h = min(tid + k * NT, HN - 1);
        const int aa = modp(A0 + h % HW - H, g.NA);
        const int bb = (D == 3) ? modp(B0 + h / HW - HB, g.NB) : 0;
        const int xs[3] = {wrap1(aa - 1, g.NA), aa, wrap1(aa + 1, g.NA)};
#pragma unroll
        for (int c = 0; c < 3; ++c) xc[k][c] = (xs[c] >> 5) * (int)Fmt<Q, S>::CHUNK + (xs[c] & 31) * Fmt<Q, S>::ESZ;
        yb[k][0] = (D == 3) ? wrap1(bb - 1, g.NB) : 0;
        yb[k][1] = bb;
        yb[k][2] = (D == 3) ? wrap1(bb + 1, g.NB) : 0;
    }
    const unsigned char* srcb = reinterpret_cast<const unsigned char*>(src);

    // M: moments of plane m over the two-node halo region
    auto moments_plane = [&](int m) {
        const int mm = modp(m, g.NM), slot = modp(m, 5), js = modp(m, 4);
        const int zr[3] = {wrap1(mm - 1, g.NM), mm, wrap1(mm + 1, g.NM)};
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const int h = tid + k * NT;
            if (h >= HN) break;
            T rd = T(0), ja = T(0), jb = T(0), jm = T(0), phi = T(0), psi = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const unsigned char* p =
                    srcb + ((long long)zr[1 - A::cm(i)] * g.NB + yb[k][1 - A::cb(i)]) * g.rowstride + xc[k][1 - A::ca(i)];
                T f, gp;
                if (Fmt<Q, S>::PAIRED && i > 0) Fmt<Q, S>::ld_fg(p, i, f, gp);  // one lane word
                else f = Fmt<Q, S>::ld_delta(p, 0, i), gp = Fmt<Q, S>::ld_delta(p, 1, i);
                rd += f;
                if (A::ca(i)) ja += T(A::ca(i)) * f;
                if (A::cb(i)) jb += T(A::cb(i)) * f;
                if (A::cm(i)) jm += T(A::cm(i)) * f;
                phi += gp;
                psi += Fmt<Q, S>::ld_delta(p, 2, i);
            }
            sm[slot][0][h] = Fmt<Q, S>::OFFSET ? T(1) + rd : rd;
            sm[slot][1][h] = phi;
            sm[slot][2][h] = psi;
            const int hx = h % HW, hy = h / HW;
            if (hx >= H && hx < H + TX && hy >= HB && hy < HB + TY) {
                const int t = (hy - HB) * TX + (hx - H);
                sj[js][0][t] = ja;
                sj[js][1][t] = jb;
                sj[js][2][t] = jm;
                sj[js][3][t] = rd;
            }
        }
    };

    // derivatives (lattice axes) of the three fields at moment-region node h of plane m
    auto derivs_ring = [&](int m, int h, T (&X0)[3], T (&grad)[3][3], T (&lap)[3]) {
        const int s0 = modp(m, 5);
        T gA[3], gB[3], gM[3], lp[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            X0[c] = sm[s0][c][h];
            gA[c] = gB[c] = gM[c] = lp[c] = T(0);
        }
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if (opp<Q>(i) < i) continue;
            const int sp_ = modp(m + A::cm(i), 5), sn = modp(m - A::cm(i), 5);
            const int cp = h + A::cb(i) * HW + A::ca(i), cn = h - A::cb(i) * HW - A::ca(i);
            const T w = T(Lat<Q>::w(i));
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T xpv = sm[sp_][c][cp], xnv = sm[sn][c][cn];
                const T d = w * (xpv - xnv);
                if (A::ca(i)) gA[c] += T(A::ca(i)) * d;
                if (A::cb(i)) gB[c] += T(A::cb(i)) * d;
                if (A::cm(i)) gM[c] += T(A::cm(i)) * d;
                lp[c] += w * (xpv + xnv);
            }
        }
        constexpr T wrest = T(1.0 - Lat<Q>::w(0));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            lap[c] = T(6) * (lp[c] - wrest * X0[c]);
            grad[c][0] = T(3) * gA[c];
            grad[c][1] = T(3) * (D == 3 ? gB[c] : gM[c]);
            grad[c][2] = D == 3 ? T(3) * gM[c] : T(0);
        }
    };

    // P: Pi of plane q over the one-node halo region
    auto pi_plane = [&](int q) {
        const int slot = modp(q, 3);
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const int pn = tid + k * NT;
            if (pn >= PN) break;
            const int h = (pn / PW + HB - PB) * HW + pn % PW + H - 1;  // the same node in the moment region
            T X[3], grad[3][3], lap[3], pi[NPI], mp, ms;
            derivs_ring(q, h, X, grad, lap);
            guo_node<Q, T>(P, X, grad, lap, pi, mp, ms);
#pragma unroll
            for (int c = 0; c < NPI; ++c) sp[slot][c][pn] = pi[c];
        }
    };

    constexpr bool PAIR = Fmt<Q, S>::OFFSET && !(Q == 19 && sizeof(S) == 4);
    MassSum<T, PAIR> msum;

    moments_plane(M0 - 2);
    moments_plane(M0 - 1);
    moments_plane(M0);
    moments_plane(M0 + 1);
    __syncthreads();
    pi_plane(M0 - 1);
    pi_plane(M0);
    __syncthreads();

    const int c0 = (ty + HB) * HW + tx + H;   // this thread's tile node in the moment region
    const int p0 = (ty + PB) * PW + tx + 1;   // ... and in the Pi region
    // the thread's own node: byte offsets of a-1, a, a+1 and rows b-1, b, b+1
    int xo[3], yo[3];
    {
        const int aa = modp(A0 + tx, g.NA), bb = (D == 3) ? modp(B0 + ty, g.NB) : 0;
        const int xs[3] = {wrap1(aa - 1, g.NA), aa, wrap1(aa + 1, g.NA)};
#pragma unroll
        for (int c = 0; c < 3; ++c) xo[c] = (xs[c] >> 5) * (int)Fmt<Q, S>::CHUNK + (xs[c] & 31) * Fmt<Q, S>::ESZ;
        yo[0] = (D == 3) ? wrap1(bb - 1, g.NB) : 0;
        yo[1] = bb;
        yo[2] = (D == 3) ? wrap1(bb + 1, g.NB) : 0;
    }
    for (int m = M0; m < M1; ++m) {
        moments_plane(m + 2);
        __syncthreads();
        pi_plane(m + 1);
        __syncthreads();
        if (!active) continue;

        // mu_phi, mu_psi from the node's fields and Laplacians
        T X0[3], grad[3][3], lap[3], pi0[NPI], mu_phi, mu_psi;
        derivs_ring(m, c0, X0, grad, lap);
        guo_node<Q, T>(P, X0, grad, lap, pi0, mu_phi, mu_psi);
        // F_a = -3 sum_i w_i sum_b e_ib Pi_ab(r + e_i) (lattice axes)
        T F[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int sl = modp(m + A::cm(i), 3);
            const int pn = p0 + A::cb(i) * PW + A::ca(i);
            const int e[3] = {Lat<Q>::cx(i), Lat<Q>::cy(i), Lat<Q>::cz(i)};
            const T w = T(Lat<Q>::w(i));
#pragma unroll
            for (int a = 0; a < D; ++a) {
                T sacc = T(0);
#pragma unroll
                for (int b = 0; b < D; ++b)
                    if (e[b]) sacc += T(e[b]) * sp[sl][GA::comp(a, b)][pn];
                F[a] -= w * sacc;
            }
        }
        F[0] *= T(3); F[1] *= T(3); F[2] *= T(3);
        const int t = ty * TX + tx, js = modp(m, 4);
        const T rdc = sj[js][3][t];
        const T jl[3] = {sj[js][0][t], D == 3 ? sj[js][1][t] : sj[js][2][t], D == 3 ? sj[js][2][t] : T(0)};
        if constexpr (PAIR) msum.add(rdc, X0[1], X0[2]);
        else msum.add(rho_total<Q, S>(rdc), X0[1], X0[2]);

        // pulled populations of the node at plane m (deviations where OFFSET)
        const int zr[3] = {wrap1(m - 1, g.NM), m, wrap1(m + 1, g.NM)};
        T fv[Q], gv[Q], kv[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const unsigned char* p =
                srcb + ((long long)zr[1 - A::cm(i)] * g.NB + yo[1 - A::cb(i)]) * g.rowstride + xo[1 - A::ca(i)];
            if (Fmt<Q, S>::PAIRED && i > 0) {
                Fmt<Q, S>::ld_fg(p, i, fv[i], gv[i]);
            } else {
                fv[i] = Fmt<Q, S>::ld_delta(p, 0, i);
                gv[i] = Fmt<Q, S>::ld_delta(p, 1, i);
            }
            kv[i] = Fmt<Q, S>::ld_delta(p, 2, i);
        }
        unsigned char* out =
            reinterpret_cast<unsigned char*>(dst) + ((long long)m * g.NB + yo[1]) * g.rowstride + xo[1];
        guo_collide_node<Q, S>(out, fv, gv, kv, rdc, jl, X0[1], X0[2], F, T(3) * P.gamma[0] * mu_phi,
                               T(3) * P.gamma[1] * mu_psi, P);
    }
    double mr, mp, ms;
    msum.get(mr, mp, ms);
    block_sum3(mr, mp, ms);
    if (tid == 0) {
        partials[3 * bid + 0] = mr;
        partials[3 * bid + 1] = mp;
        partials[3 * bid + 2] = ms;
    }
}

template <int Q, typename S, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, 512 / (TX * TY))
k_guo_fused(MGeom g, const S* __restrict__ src, S* __restrict__ dst, Phys<typename Store<S>::T> P,
            double* __restrict__ partials) {
    guo_body<Q, S, TX, TY>(g, src, dst, P, partials, blockIdx.x);
}

// One step of the forcing coupling with the marching kernel (tile from fused_cfg).
template <int Q, typename S>
inline cudaError_t guo_fused_step(tlbm_host::DevState& d, const Phys<typename Store<S>::T>& P, cudaStream_t st) {
    const FusedCfg<Q> c = fused_cfg<Q>(d);
    const MGeom g = mgeom<Q, S>(d, c);
    const long long nb = (long long)g.tilesA * g.tilesB * g.NC;
    if (nb > 0x7fffffffLL || nb > d.partials_cap) return cudaErrorInvalidConfiguration;
    const S* src = static_cast<const S*>(d.pop[d.cur]);
    S* dst = static_cast<S*>(d.pop[1 - d.cur]);
    if constexpr (Q == 19) {
        if constexpr (sizeof(S) == 8) k_guo_fused<Q, S, 16, 4><<<(int)nb, 64, 0, st>>>(g, src, dst, P, d.partials);
        else k_guo_fused<Q, S, 32, 4><<<(int)nb, 128, 0, st>>>(g, src, dst, P, d.partials);
    } else {
        k_guo_fused<Q, S, 128, 1><<<(int)nb, 128, 0, st>>>(g, src, dst, P, d.partials);
    }
    return cudaGetLastError();
}

}  // namespace tlbm_dev
