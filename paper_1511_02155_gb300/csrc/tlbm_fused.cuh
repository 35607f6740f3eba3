// tlbm_fused.cuh -- one-kernel time step of the ternary free-energy LB method
// (Semprebon, Krueger, Kusumaatmaja, arXiv:1511.02155) for periodic lattices
// without solid nodes.
//
// The equilibria at r need gradients and Laplacians of rho, phi, psi at the
// same time level, i.e. the moments of r's neighbours, which depend on the
// neighbours' populations.  Instead of writing moment arrays to HBM and
// reading the populations twice, each block owns a column of the lattice
// (a TX x TY tile of the in-plane axes) and marches along the last axis
// (z for D3Q19, y for D2Q9) over a chunk of MC planes:
//
//   prologue: moments of planes m0-1 and m0 (tile + one-node halo) -> smem
//   for each plane m of the chunk:
//     M: pull populations of plane m+1 over tile + halo, reduce them to
//        rho, phi, psi (and j = rho u on the tile) into a shared ring
//     __syncthreads
//     C: for each tile node of plane m: gradients and Laplacians from the
//        ring (planes m-1, m, m+1), local thermodynamics, equilibria,
//        BGK, and the store of x*(r) -- populations are pulled again
//        (L1/L2 hits: phase M read them one iteration earlier).
//
// The moment ring has four slots and the j ring three, so one barrier per
// plane suffices (a fast warp writing plane m+2 never touches a slot that a
// slow warp still reads for plane m).  HBM traffic per node is one read and one
// write of the 3Q populations plus the halo's share (about 2/MC extra planes).
#pragma once

#include "tlbm_kernels.cuh"

namespace tlbm_dev {

// velocity components in (in-plane a, in-plane b, marching m) coordinates
template <int Q>
struct Axes {
    static constexpr int D = Lat<Q>::D;
    __host__ __device__ static constexpr int ca(int i) { return Lat<Q>::cx(i); }
    __host__ __device__ static constexpr int cb(int i) { return D == 3 ? Lat<Q>::cy(i) : 0; }
    __host__ __device__ static constexpr int cm(int i) { return D == 3 ? Lat<Q>::cz(i) : Lat<Q>::cy(i); }
};

struct MGeom {
    int NA, NB, NM;       // extents along a, b, m
    long long plane;      // NA * NB
    long long Np;         // direction stride
    int MC;               // planes per chunk
    int tilesA, tilesB;   // tiles per plane
};

__device__ __forceinline__ int modp(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

template <int Q, typename S, int TX, int TY>
__global__ void __launch_bounds__(TX * TY)
k_fused(MGeom g, const S* __restrict__ src, S* __restrict__ dst, Phys<typename Store<S>::T> P,
        double* __restrict__ partials) {
    using T = typename Store<S>::T;
    using A = Axes<Q>;
    constexpr int D = Lat<Q>::D;
    constexpr int HY = (D == 3) ? 1 : 0;  // halo rows along b
    constexpr int HW = TX + 2;
    constexpr int HH = TY + 2 * HY;
    constexpr int HN = HW * HH;
    constexpr int NT = TX * TY;
    static_assert(D == 3 || TY == 1, "2-D tiles are one row");

    __shared__ T sm[4][3][HN];  // moment ring: rho, phi, psi over tile + halo
    __shared__ T sj[3][3][NT];  // j ring over the tile

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int tileA = blockIdx.x % g.tilesA;
    const int rest = blockIdx.x / g.tilesA;
    const int tileB = rest % g.tilesB;
    const int chunk = rest / g.tilesB;
    const int A0 = tileA * TX, B0 = tileB * TY;
    const int M0 = chunk * g.MC;
    const int M1 = min(M0 + g.MC, g.NM);
    const int a = A0 + tx, b = B0 + ty;
    const bool active = (a < g.NA) && (b < g.NB);

    // Phase M: moments of plane m over tile + halo into ring slot `slot`.
    auto moments_plane = [&](int m, int slot, int jslot) {
        const int mm = modp(m, g.NM);
        const long long om[3] = {(long long)modp(mm - 1, g.NM) * g.plane, (long long)mm * g.plane,
                                 (long long)modp(mm + 1, g.NM) * g.plane};
        for (int h = tid; h < HN; h += NT) {
            const int hx = h % HW, hy = h / HW;
            const int aa = modp(A0 + hx - 1, g.NA);
            const int bb = (D == 3) ? modp(B0 + hy - HY, g.NB) : 0;
            const long long oa[3] = {modp(aa - 1, g.NA), aa, modp(aa + 1, g.NA)};
            const long long ob[3] = {(long long)modp(bb - 1, g.NB) * g.NA, (long long)bb * g.NA,
                                     (long long)modp(bb + 1, g.NB) * g.NA};
            T rho = T(0), ja = T(0), jb = T(0), jm = T(0), phi = T(0), psi = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const long long q = oa[1 - A::ca(i)] + ob[1 - A::cb(i)] + om[1 - A::cm(i)];
                const T f = Store<S>::ld(src, (long long)(0 * Q + i) * g.Np + q, T(rest_offset<Q, S>(0, i)));
                rho += f;
                if (A::ca(i)) ja += T(A::ca(i)) * f;
                if (A::cb(i)) jb += T(A::cb(i)) * f;
                if (A::cm(i)) jm += T(A::cm(i)) * f;
                phi += Store<S>::ld(src, (long long)(1 * Q + i) * g.Np + q, T(0));
                psi += Store<S>::ld(src, (long long)(2 * Q + i) * g.Np + q, T(0));
            }
            sm[slot][0][h] = rho;
            sm[slot][1][h] = phi;
            sm[slot][2][h] = psi;
            if (jslot >= 0 && hx >= 1 && hx <= TX && hy >= HY && hy < HY + TY) {
                const int t = (hy - HY) * TX + (hx - 1);
                sj[jslot][0][t] = ja;
                sj[jslot][1][t] = jb;
                sj[jslot][2][t] = jm;
            }
        }
    };

    double mr = 0.0, mp = 0.0, ms = 0.0;

    moments_plane(M0 - 1, (M0 + 3) & 3, -1);
    moments_plane(M0, M0 & 3, M0 % 3);

    const long long oa_c[3] = {modp(a - 1, g.NA), a, modp(a + 1, g.NA)};
    const long long ob_c[3] = {(long long)modp(b - 1, g.NB) * g.NA, (long long)b * g.NA,
                               (long long)modp(b + 1, g.NB) * g.NA};

    for (int m = M0; m < M1; ++m) {
        moments_plane(m + 1, (m + 1) & 3, (m + 1) % 3);
        __syncthreads();
        if (!active) continue;

        // ---- derivatives from the ring (pairs of opposite links)
        const int hx0 = tx + 1, hy0 = ty + HY;
        const int c0 = hy0 * HW + hx0;
        T X0[3], gA[3], gB[3], gM[3], lp[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            X0[c] = sm[m & 3][c][c0];
            gA[c] = gB[c] = gM[c] = lp[c] = T(0);
        }
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if (opp<Q>(i) < i) continue;
            const int sp = (m + A::cm(i)) & 3, sn = (m - A::cm(i)) & 3;
            const int cp = c0 + A::cb(i) * HW + A::ca(i);
            const int cn = c0 - A::cb(i) * HW - A::ca(i);
            const T w = T(Lat<Q>::w(i));
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T xp = sm[sp][c][cp], xn = sm[sn][c][cn];
                const T d = w * (xp - xn);
                if (A::ca(i)) gA[c] += T(A::ca(i)) * d;
                if (A::cb(i)) gB[c] += T(A::cb(i)) * d;
                if (A::cm(i)) gM[c] += T(A::cm(i)) * d;
                lp[c] += w * (xp + xn);
            }
        }
        T grad[3][3], lap[3];
        constexpr T wrest = T(1.0 - Lat<Q>::w(0));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            lap[c] = T(6) * (lp[c] - wrest * X0[c]);
            grad[c][0] = T(3) * gA[c];
            if (D == 3) {
                grad[c][1] = T(3) * gB[c];
                grad[c][2] = T(3) * gM[c];
            } else {
                grad[c][1] = T(3) * gM[c];
                grad[c][2] = T(0);
            }
        }
        const int t = ty * TX + tx;
        const int js = m % 3;
        const T jA = sj[js][0][t], jB = sj[js][1][t], jM = sj[js][2][t];
        NodeEq<Q, T> E;
        if (D == 3) E.setup(P, X0[0], jA, jB, jM, X0[1], X0[2], grad, lap);
        else E.setup(P, X0[0], jA, jM, T(0), X0[1], X0[2], grad, lap);
        mr += (double)X0[0]; mp += (double)X0[1]; ms += (double)X0[2];

        // ---- collide + store, direction pairs
        const long long om_c[3] = {(long long)modp(m - 1, g.NM) * g.plane, (long long)m * g.plane,
                                   (long long)modp(m + 1, g.NM) * g.plane};
        const long long r = oa_c[1] + ob_c[1] + om_c[1];
        T sf = T(0), sg = T(0), sk = T(0);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int o = opp<Q>(i);
            if (o < i) continue;
            const long long qi = oa_c[1 - A::ca(i)] + ob_c[1 - A::cb(i)] + om_c[1 - A::cm(i)];
            const long long qo = oa_c[1 + A::ca(i)] + ob_c[1 + A::cb(i)] + om_c[1 + A::cm(i)];
            const T offi = T(rest_offset<Q, S>(0, i));
            const T fi = Store<S>::ld(src, (long long)(0 * Q + i) * g.Np + qi, offi);
            const T fo = Store<S>::ld(src, (long long)(0 * Q + o) * g.Np + qo, offi);
            const T gi = Store<S>::ld(src, (long long)(1 * Q + i) * g.Np + qi, T(0));
            const T go = Store<S>::ld(src, (long long)(1 * Q + o) * g.Np + qo, T(0));
            const T ki = Store<S>::ld(src, (long long)(2 * Q + i) * g.Np + qi, T(0));
            const T ko = Store<S>::ld(src, (long long)(2 * Q + o) * g.Np + qo, T(0));
            // equilibria of the pair: even part shared, odd part flips sign
            const T w = T(Lat<Q>::w(i));
            const T e = E.eu(i);
            const T e2 = T(4.5) * e * e;
            const T gt = E.grad_term(i);
            const T fev = w * (E.bf + E.rho * e2) + gt, fod = w * T(3) * E.rho * e;
            const T gev = w * (E.bg + E.phi * e2), god = w * T(3) * E.phi * e;
            const T kev = w * (E.bk + E.psi * e2), kod = w * T(3) * E.psi * e;
            sf += T(2) * fev; sg += T(2) * gev; sk += T(2) * kev;
            Store<S>::st(dst, (long long)(0 * Q + i) * g.Np + r, fi + P.omega[0] * ((fev + fod) - fi), offi);
            Store<S>::st(dst, (long long)(0 * Q + o) * g.Np + r, fo + P.omega[0] * ((fev - fod) - fo), offi);
            Store<S>::st(dst, (long long)(1 * Q + i) * g.Np + r, gi + P.omega[1] * ((gev + god) - gi), T(0));
            Store<S>::st(dst, (long long)(1 * Q + o) * g.Np + r, go + P.omega[1] * ((gev - god) - go), T(0));
            Store<S>::st(dst, (long long)(2 * Q + i) * g.Np + r, ki + P.omega[2] * ((kev + kod) - ki), T(0));
            Store<S>::st(dst, (long long)(2 * Q + o) * g.Np + r, ko + P.omega[2] * ((kev - kod) - ko), T(0));
        }
        const T off0 = T(rest_offset<Q, S>(0, 0));
        const T f0 = Store<S>::ld(src, r, off0);
        const T g0 = Store<S>::ld(src, (long long)Q * g.Np + r, T(0));
        const T k0 = Store<S>::ld(src, (long long)2 * Q * g.Np + r, T(0));
        Store<S>::st(dst, r, f0 + P.omega[0] * ((E.rho - sf) - f0), off0);
        Store<S>::st(dst, (long long)Q * g.Np + r, g0 + P.omega[1] * ((E.phi - sg) - g0), T(0));
        Store<S>::st(dst, (long long)2 * Q * g.Np + r, k0 + P.omega[2] * ((E.psi - sk) - k0), T(0));
    }

    block_sum3(mr, mp, ms);
    if (tid == 0) {
        partials[3 * blockIdx.x + 0] = mr;
        partials[3 * blockIdx.x + 1] = mp;
        partials[3 * blockIdx.x + 2] = ms;
    }
}

// ------------------------------------------------------------ host side

// tile variants: 0 = default for the lattice; D3Q19: 1 = 32x8, 2 = 64x4, 3 = 16x16;
// D2Q9: 1 = 128, 2 = 256, 3 = 64.  tile = variant + 16 * chunk (chunk 0 = auto).
template <int Q>
struct FusedCfg {
    int TX, TY, MC;
};

template <int Q>
inline FusedCfg<Q> fused_cfg(const tlbm_host::DevState& d) {
    const int variant = d.prec == 0 ? 0 : (d.tile & 15);  // double storage: default tile only
    int mc = d.tile >> 4;
    FusedCfg<Q> c{};
    if (Q == 19 && d.prec == 0) {
        c.TX = 16;  // double storage: a smaller tile keeps the static shared ring under 48 KB
        c.TY = 8;
    } else if (Q == 19) {
        const int v = variant == 0 ? 1 : variant;
        c.TX = v == 2 ? 64 : (v == 3 ? 16 : 32);
        c.TY = v == 2 ? 4 : (v == 3 ? 16 : 8);
    } else {
        const int v = variant == 0 ? 1 : variant;
        c.TX = v == 2 ? 256 : (v == 3 ? 64 : 128);
        c.TY = 1;
    }
    const int NA = d.nx;
    const int NB = (Q == 19) ? d.ny : 1;
    const int NM = (Q == 19) ? d.nz : d.ny;
    if (mc <= 0) {
        // enough blocks to fill 152 SMs a few times over, chunks of at most 64 planes
        const long long cols = (long long)((NA + c.TX - 1) / c.TX) * ((NB + c.TY - 1) / c.TY);
        mc = 64;
        while (mc > 4 && cols * ((NM + mc - 1) / mc) < 4 * 152) mc >>= 1;
    }
    c.MC = mc < 1 ? 1 : (mc > NM ? NM : mc);
    return c;
}

template <int Q, typename S>
inline bool fused_supported(const tlbm_host::DevState& d) {
    return d.solid == nullptr;
}

template <int Q, typename S>
inline int fused_launches(const tlbm_host::DevState&) {
    return 1;
}

template <int Q>
inline MGeom mgeom(const tlbm_host::DevState& d, const FusedCfg<Q>& c) {
    MGeom g;
    g.NA = d.nx;
    g.NB = (Q == 19) ? d.ny : 1;
    g.NM = (Q == 19) ? d.nz : d.ny;
    g.plane = (long long)g.NA * g.NB;
    g.Np = d.Np;
    g.MC = c.MC;
    g.tilesA = (g.NA + c.TX - 1) / c.TX;
    g.tilesB = (g.NB + c.TY - 1) / c.TY;
    return g;
}

template <int Q>
inline long long fused_blocks(const tlbm_host::DevState& d) {
    const FusedCfg<Q> c = fused_cfg<Q>(d);
    const MGeom g = mgeom<Q>(d, c);
    return (long long)g.tilesA * g.tilesB * ((g.NM + g.MC - 1) / g.MC);
}

// number of partial sums the last step wrote (for k_mass_final)
template <int Q, typename S>
inline int fused_partials(const tlbm_host::DevState& d, int kind) {
    return kind == tlbm_host::KIND_FUSED ? (int)fused_blocks<Q>(d) : kMassBlocks;
}

template <int Q, typename S>
inline cudaError_t fused_step(tlbm_host::DevState& d, const Phys<typename Store<S>::T>& P, cudaStream_t st) {
    const FusedCfg<Q> c = fused_cfg<Q>(d);
    const MGeom g = mgeom<Q>(d, c);
    const long long nb = (long long)g.tilesA * g.tilesB * ((g.NM + g.MC - 1) / g.MC);
    if (nb > 0x7fffffffLL || nb > d.partials_cap) return cudaErrorInvalidConfiguration;
    const S* src = static_cast<const S*>(d.pop[d.cur]);
    S* dst = static_cast<S*>(d.pop[1 - d.cur]);
    if constexpr (sizeof(S) == 8) {
        // double storage is the parity path: one tile shape per lattice
        if constexpr (Q == 19) k_fused<Q, S, 16, 8><<<(int)nb, 128, 0, st>>>(g, src, dst, P, d.partials);
        else k_fused<Q, S, 128, 1><<<(int)nb, 128, 0, st>>>(g, src, dst, P, d.partials);
    } else if constexpr (Q == 19) {
        if (c.TX == 64) k_fused<Q, S, 64, 4><<<(int)nb, 256, 0, st>>>(g, src, dst, P, d.partials);
        else if (c.TX == 16) k_fused<Q, S, 16, 16><<<(int)nb, 256, 0, st>>>(g, src, dst, P, d.partials);
        else k_fused<Q, S, 32, 8><<<(int)nb, 256, 0, st>>>(g, src, dst, P, d.partials);
    } else {
        if (c.TX == 256) k_fused<Q, S, 256, 1><<<(int)nb, 256, 0, st>>>(g, src, dst, P, d.partials);
        else if (c.TX == 64) k_fused<Q, S, 64, 1><<<(int)nb, 64, 0, st>>>(g, src, dst, P, d.partials);
        else k_fused<Q, S, 128, 1><<<(int)nb, 128, 0, st>>>(g, src, dst, P, d.partials);
    }
    return cudaGetLastError();
}

}  // namespace tlbm_dev
