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

#include <vector>

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
    int NC;               // chunks along m; chunk c holds planes [c NM / NC, (c+1) NM / NC)
    int tilesA, tilesB;   // tiles per plane
    long long rowstride;  // bytes between consecutive (b, m) rows: ncx * chunk bytes
    long long bytes;      // bytes of one population buffer (bounds-checked kernels)
    unsigned long long* check;  // first bounds violation (bounds-checked kernels)
};

// Bounds checks of the checked kernel variants (CHK).  A violation is recorded
// as (code << 56 | offset) in *g.check -- the first one wins -- and the access
// is redirected to a valid address; nothing traps.  Codes: 1 pull source,
// 2 bounce-back source, 3 store target, 4 moment-ring index, 5 mask index.
__device__ __forceinline__ void chk_record(const MGeom& g, unsigned code, long long v) {
    atomicCAS(g.check, 0ull, ((unsigned long long)code << 56) | ((unsigned long long)v & 0x00ffffffffffffffull));
}
// a node pointer (chunk + lane * ESZ) of a population buffer starting at base
template <int Q, typename S, bool CHK, typename P>
__device__ __forceinline__ P* chk_node(const MGeom& g, P* base, P* p, unsigned code) {
    if constexpr (CHK) {
        const long long off = (const unsigned char*)p - (const unsigned char*)base;
        if (off < 0 || off >= g.bytes || (off % Fmt<Q, S>::CHUNK) >= 32LL * Fmt<Q, S>::ESZ) {
            chk_record(g, code, off);
            return base;
        }
    }
    return p;
}
// an index into an array of n entries
template <bool CHK>
__device__ __forceinline__ long long chk_index(const MGeom& g, long long i, long long n, unsigned code) {
    if constexpr (CHK) {
        if (i < 0 || i >= n) {
            chk_record(g, code, i);
            return 0;
        }
    }
    return i;
}

__device__ __forceinline__ int modp(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// single periodic wrap of v in [-n, 2n)
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }


// L2 bulk prefetch (TMA unit) of [p, p + bytes); p 16-byte aligned, bytes a
// multiple of 16.  A hint: it does not fault and does not wait.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ILP: a thread's border node loads interleave with its own node's loads.
// EARLY: phase C's loads are issued before phase M's (values held across M).
// PF: each warp prefetches its own 32-node chunk three planes ahead into L2.
// HINT: 1 streams the stores out (evict-first); 2 also marks phase C's loads,
//       the last use of those lines, evict-first.
// STG: STG of the 3Q pulled populations of a thread's own node, loaded in
//      phase M, are kept in shared memory (2 plane slots x STG x NT values) and
//      the collision reads them from there instead of pulling them again from
//      L2; stage_rank orders the candidates (STGO 0: the lane-shifted
//      directions first, whose warp loads span two chunks; 1: set by set).
// position of population (s, i) in the staging order: STGO 1 set by set; STGO 0
// the lane-shifted directions (e_x != 0) of all three sets first
template <int Q, int STGO>
__host__ __device__ constexpr int stage_rank(int s, int i) {
    if (STGO == 1) return s * Q + i;
    if (Q == 19) {
        const bool sh = (i == 1 || i == 2) || (i >= 7 && i <= 10) || (i >= 15);
        const int is = i <= 2 ? i - 1 : (i <= 10 ? i - 5 : i - 9);
        const int iu = i == 0 ? 0 : (i <= 6 ? i - 2 : i - 6);
        if (STGO == 2) {
            // paired lane words: the k values first (each a lone value of its
            // word), lane-shifted first; then the lane-shifted (f, g) pairs; then
            // the other pairs and the rest populations
            if (i == 0) return 54 + s;
            if (s == 2) return sh ? is : 10 + iu - 1;
            return 18 + (sh ? 2 * is + s : 20 + 2 * (iu - 1) + s);
        }
        return sh ? s * 10 + is : 30 + s * 9 + iu;
    }
    const bool sh = i == 1 || i == 2 || i >= 5;
    const int is = i <= 2 ? i - 1 : i - 3;
    const int iu = i == 0 ? 0 : i - 2;
    return sh ? s * 6 + is : 18 + s * 3 + iu;
}

// Mass totals (rho, phi, psi of the step's input state) of the nodes a thread
// collides, given rd (rho, or rho - 1 where f is stored as f_i - w_i), phi, psi.
// PAIR false sums in double, as the other kernels do.  PAIR true (float
// formats) keeps per quantity an error-free pair (hi, lo) updated by Knuth's
// TwoSum, and rho as the node count plus the summed deviations: no FP64
// instruction runs per node, and the pairs become doubles once per block.
// Measured on GB300: the pairs are 1-2 % faster for D2Q9 and for 16-bit D3Q19
// storage; the FP32 D3Q19 kernel, at its register limit, spills with them and
// keeps the double sums.
template <typename T, bool PAIR>
struct MassSum {
    double r = 0.0, p = 0.0, s = 0.0;
    __device__ __forceinline__ void add(double rho, T phi, T psi) {  // rho: rho_total of rd
        r += rho;
        p += (double)phi;
        s += (double)psi;
    }
    __device__ __forceinline__ void get(double& a, double& b, double& c) const {
        a = r;
        b = p;
        c = s;
    }
};
template <>
struct MassSum<float, true> {
    float h[3] = {0.0f, 0.0f, 0.0f}, l[3] = {0.0f, 0.0f, 0.0f};
    int n = 0;
    __device__ __forceinline__ void acc(int c, float x) {
        const float sum = h[c] + x;
        const float bp = sum - h[c];
        l[c] += (h[c] - (sum - bp)) + (x - bp);  // the rounding error of h + x, exactly
        h[c] = sum;
    }
    __device__ __forceinline__ void add(float rd, float phi, float psi) {  // rd = rho - 1 (offset formats)
        acc(0, rd);
        acc(1, phi);
        acc(2, psi);
        ++n;
    }
    __device__ __forceinline__ void get(double& a, double& b, double& c) const {
        a = (double)n + ((double)h[0] + (double)l[0]);
        b = (double)h[1] + (double)l[1];
        c = (double)h[2] + (double)l[2];
    }
};

// FP32 load through the non-coherent path with an L2 fetch size of 256 bytes:
// a miss brings the neighbouring 128-byte run of the chunk into L2 as well.
__device__ __forceinline__ float ld_l2x256(const unsigned char* p) {
    float v;
    asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

template <int Q, typename S, int TX, int TY, bool ILP, bool EARLY, bool PF = false, int HINT = 0, int STG = 0,
          int STGO = 1, bool CHK = false, int LDH = 0>
__device__ __forceinline__ void fused_body(const MGeom& g, const S* __restrict__ src, S* __restrict__ dst,
                                           const Phys<typename Store<S>::T>& P, double* __restrict__ partials,
                                           const int bid) {
    using T = typename Store<S>::T;
    using A = Axes<Q>;
    // staging ring in dynamic shared memory (declared here so that the compiler
    // knows the stores are shared-memory stores that cannot alias the loads)
    extern __shared__ __align__(16) unsigned char tlbm_stage_smem[];
    T* const stg = reinterpret_cast<T*>(tlbm_stage_smem);
    constexpr int D = Lat<Q>::D;
    constexpr int HY = (D == 3) ? 1 : 0;  // halo rows along b
    constexpr int HW = TX + 2;
    constexpr int HH = TY + 2 * HY;
    constexpr int HN = HW * HH;
    constexpr int NT = TX * TY;
    constexpr int NBORDER = HN - NT;
    static_assert(D == 3 || TY == 1, "2-D tiles are one row");
    static_assert(NBORDER <= NT, "one border node per thread at most");

    __shared__ T sm[4][3][HN];  // moment ring: rho, phi, psi over tile + halo

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

    // Node 0 of every thread: its own tile slot (coordinates wrap for threads past
    // the lattice edge, whose slots serve as the periodic halo of active ones).
    // Node 1: one border slot of the halo ring, for tid < NBORDER.
    int h[2], xc[2][3], yb[2][3];  // ring slot; byte offsets of x-1, x, x+1 in a row; rows b-1, b, b+1
    {
        int hx[2], hy[2];
        hx[0] = tx + 1;
        hy[0] = ty + HY;
        hx[1] = 0;
        hy[1] = 0;
        if (D == 2) {
            hx[1] = tid == 0 ? 0 : HW - 1;
        } else if (tid < HW) {
            hx[1] = tid;
        } else if (tid < 2 * HW) {
            hx[1] = tid - HW;
            hy[1] = HH - 1;
        } else if (tid < NBORDER) {
            const int k = tid - 2 * HW;
            hx[1] = k < HH - 2 ? 0 : HW - 1;
            hy[1] = 1 + (k < HH - 2 ? k : k - (HH - 2));
        } else {  // no border node: node 1 repeats node 0 (never used)
            hx[1] = hx[0];
            hy[1] = hy[0];
        }
#pragma unroll
        for (int n = 0; n < 2; ++n) {
            h[n] = (int)chk_index<CHK>(g, hy[n] * HW + hx[n], HN, 4);
            const int aa = modp(A0 + hx[n] - 1, g.NA);
            const int bb = (D == 3) ? modp(B0 + hy[n] - HY, g.NB) : 0;
            const int xs[3] = {wrap1(aa - 1, g.NA), aa, wrap1(aa + 1, g.NA)};
#pragma unroll
            for (int k = 0; k < 3; ++k) xc[n][k] = (xs[k] >> 5) * (int)Fmt<Q, S>::CHUNK + (xs[k] & 31) * Fmt<Q, S>::ESZ;
            yb[n][0] = (D == 3) ? wrap1(bb - 1, g.NB) : 0;
            yb[n][1] = bb;
            yb[n][2] = (D == 3) ? wrap1(bb + 1, g.NB) : 0;
        }
    }
    const int nnodes = tid < NBORDER ? 2 : 1;

    const unsigned char* srcb = reinterpret_cast<const unsigned char*>(src);
    // stored value (x - bias) of (s, i) at node pointer p (LDH 1, FP32: with the
    // 256-byte L2 fetch hint)
    auto ldp = [&](const unsigned char* p, int s, int i) -> T {
        if constexpr (LDH == 1 && sizeof(S) == 4) return ld_l2x256(p + Fmt<Q, S>::off(s, i));
        else return Fmt<Q, S>::ld_delta(p, s, i);
    };
    // pull source of direction (ca, cb, cm) for node n at plane rows zr
    auto src_of = [&](int n, const int (&zr)[3], int ca, int cb, int cm) -> const unsigned char* {
        const long long row = (long long)zr[1 - cm] * g.NB + yb[n][1 - cb];
        return chk_node<Q, S, CHK>(g, srcb, srcb + row * g.rowstride + xc[n][1 - ca], 1);
    };

    // Phase M: moments of plane m for this thread's nodes into ring slot `slot`;
    // node 0's momentum density is returned in j and its summed f deviations
    // (rho - 1 in the 16-bit formats, rho otherwise) in rd.
    auto moments_plane = [&](int m, int slot, T (&j)[3], T& rd) {
        const int mm = wrap1(m, g.NM);
        const int zr[3] = {wrap1(mm - 1, g.NM), mm, wrap1(mm + 1, g.NM)};
        const bool two = nnodes == 2;
        T rho0 = T(0), ja = T(0), jb = T(0), jm = T(0), phi0 = T(0), psi0 = T(0);
        T rho1 = T(0), phi1 = T(0), psi1 = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const unsigned char* p0 = src_of(0, zr, A::ca(i), A::cb(i), A::cm(i));
            T f, gg;
            if (Fmt<Q, S>::PAIRED && i > 0) Fmt<Q, S>::ld_fg(p0, i, f, gg);  // one lane word
            else f = ldp(p0, 0, i), gg = ldp(p0, 1, i);
            const T kk = ldp(p0, 2, i);
            rho0 += f;
            if (A::ca(i)) ja += T(A::ca(i)) * f;
            if (A::cb(i)) jb += T(A::cb(i)) * f;
            if (A::cm(i)) jm += T(A::cm(i)) * f;
            phi0 += gg;
            psi0 += kk;
            if constexpr (STG > 0) {
                T* sp = stg + (size_t)((m & 1) * STG) * NT + tid;
                const int r0 = stage_rank<Q, STGO>(0, i), r1 = stage_rank<Q, STGO>(1, i),
                              r2 = stage_rank<Q, STGO>(2, i);
                if (r0 < STG) sp[(size_t)r0 * NT] = f;
                if (r1 < STG) sp[(size_t)r1 * NT] = gg;
                if (r2 < STG) sp[(size_t)r2 * NT] = kk;
            }
            if (ILP && two) {  // border node of this thread, loads interleaved with node 0
                const unsigned char* p1 = src_of(1, zr, A::ca(i), A::cb(i), A::cm(i));
                if (Fmt<Q, S>::PAIRED && i > 0) {
                    T a, b;
                    Fmt<Q, S>::ld_fg(p1, i, a, b);
                    rho1 += a;
                    phi1 += b;
                } else {
                    rho1 += ldp(p1, 0, i);
                    phi1 += ldp(p1, 1, i);
                }
                psi1 += ldp(p1, 2, i);
            }
        }
        if (!ILP && two) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const unsigned char* p1 = src_of(1, zr, A::ca(i), A::cb(i), A::cm(i));
                if (Fmt<Q, S>::PAIRED && i > 0) {
                    T a, b;
                    Fmt<Q, S>::ld_fg(p1, i, a, b);
                    rho1 += a;
                    phi1 += b;
                } else {
                    rho1 += ldp(p1, 0, i);
                    phi1 += ldp(p1, 1, i);
                }
                psi1 += ldp(p1, 2, i);
            }
        }
        rd = rho0;
        if (Fmt<Q, S>::OFFSET) {  // sums of f deviations: rho - 1
            rho0 += T(1);
            rho1 += T(1);
        }
        sm[slot][0][h[0]] = rho0;
        sm[slot][1][h[0]] = phi0;
        sm[slot][2][h[0]] = psi0;
        if (two) {
            sm[slot][0][h[1]] = rho1;
            sm[slot][1][h[1]] = phi1;
            sm[slot][2][h[1]] = psi1;
        }
        j[0] = ja;
        j[1] = jb;
        j[2] = jm;
    };

    constexpr bool PAIR = Fmt<Q, S>::OFFSET && !(Q == 19 && sizeof(S) == 4);
    MassSum<T, PAIR> msum;
    T jc[3], jn[3], rdc, rdn;

    moments_plane(M0 - 1, (M0 + 3) & 3, jn, rdn);
    moments_plane(M0, M0 & 3, jc, rdc);

    for (int m = M0; m < M1; ++m) {
        // Pulled populations of this thread's node at plane m, loaded before the
        // phase-M loads of plane m+1 so that both sets of requests are in flight
        // together (these were read one iteration ago and hit in L2).
        const int zr[3] = {wrap1(m - 1, g.NM), m, wrap1(m + 1, g.NM)};
        // stored values (deviations x - bias: the 16-bit formats keep f as f_i - w_i;
        // the collision below works on deviations, with the bias folded into its
        // constants)
        T fv[Q], gv[Q], kv[Q];
        auto load_node = [&]() {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const unsigned char* pi = src_of(0, zr, A::ca(i), A::cb(i), A::cm(i));
                auto lc = [&](int s_) -> T {
                    return HINT >= 2 ? Fmt<Q, S>::ld_last_delta(pi, s_, i) : Fmt<Q, S>::ld_delta(pi, s_, i);
                };
                if constexpr (STG > 0) {
                    const T* sp = stg + (size_t)((m & 1) * STG) * NT + tid;
                    const int r0 = stage_rank<Q, STGO>(0, i), r1 = stage_rank<Q, STGO>(1, i),
                              r2 = stage_rank<Q, STGO>(2, i);
                    if (Fmt<Q, S>::PAIRED && i > 0 && r0 >= STG && r1 >= STG) {
                        Fmt<Q, S>::template ld_fg<(HINT >= 2)>(pi, i, fv[i], gv[i]);  // one lane word
                    } else {
                        fv[i] = r0 < STG ? sp[(size_t)r0 * NT] : lc(0);
                        gv[i] = r1 < STG ? sp[(size_t)r1 * NT] : lc(1);
                    }
                    kv[i] = r2 < STG ? sp[(size_t)r2 * NT] : lc(2);
                } else {
                    if (Fmt<Q, S>::PAIRED && i > 0) {
                        Fmt<Q, S>::template ld_fg<(HINT >= 2)>(pi, i, fv[i], gv[i]);
                    } else {
                        fv[i] = lc(0);
                        gv[i] = lc(1);
                    }
                    kv[i] = lc(2);
                }
            }
        };
        if (EARLY && active) load_node();
        if (PF && (tid & 31) == 0 && active && m + 3 <= M1 + 1) {
            // this warp's chunk of plane m+3 (all populations of its 32 nodes)
            const long long row = (long long)wrap1(m + 3 >= g.NM ? m + 3 - g.NM : m + 3, g.NM) * g.NB + yb[0][1];
            prefetch_l2(srcb + row * g.rowstride + xc[0][1] - ((A0 + tx) & 31) * Fmt<Q, S>::ESZ,
                        (unsigned)Fmt<Q, S>::CHUNK);
        }
        moments_plane(m + 1, (m + 1) & 3, jn, rdn);
        __syncthreads();
        if (active) {
            if (!EARLY) load_node();
            // ---- derivatives from the ring (pairs of opposite links)
            const int c0 = h[0];
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
                const int cp = (int)chk_index<CHK>(g, c0 + A::cb(i) * HW + A::ca(i), HN, 4);
                const int cn = (int)chk_index<CHK>(g, c0 - A::cb(i) * HW - A::ca(i), HN, 4);
                const T w = T(Lat<Q>::w(i));
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const T xpv = sm[sp][c][cp], xnv = sm[sn][c][cn];
                    const T d = w * (xpv - xnv);
                    if (A::ca(i)) gA[c] += T(A::ca(i)) * d;
                    if (A::cb(i)) gB[c] += T(A::cb(i)) * d;
                    if (A::cm(i)) gM[c] += T(A::cm(i)) * d;
                    lp[c] += w * (xpv + xnv);
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
            NodeEq<Q, T> E;
            if (D == 3) E.setup(P, X0[0], jc[0], jc[1], jc[2], X0[1], X0[2], grad, lap, rdc);
            else E.setup(P, X0[0], jc[0], jc[2], T(0), X0[1], X0[2], grad, lap, rdc);
            if constexpr (PAIR) msum.add(rdc, X0[1], X0[2]);
            else msum.add(rho_total<Q, S>(rdc), X0[1], X0[2]);

            // ---- collide + store, direction pairs
            unsigned char* out = chk_node<Q, S, CHK>(
                g, reinterpret_cast<unsigned char*>(dst),
                reinterpret_cast<unsigned char*>(dst) + ((long long)m * g.NB + yb[0][1]) * g.rowstride + xc[0][1], 3);

            auto st_ = [&](unsigned char* o, int ss, int ii, T d) {
                if (HINT >= 1) Fmt<Q, S>::st_stream_delta(o, ss, ii, d);
                else Fmt<Q, S>::st_delta(o, ss, ii, d);
            };
            // BGK with omega folded into the equilibria: x* = (1 - omega) x + omega x_eq,
            // and omega x_eq = EV +- OD for a pair of opposite links, where
            // EV = w (B + R (e.u)^2) [+ gradient terms for f] and OD = w O (e.u).
            // On deviations d = x - w b (b = 1 for f in the offset formats, else 0):
            // d* = (1 - omega) d + EV - omega w b +- OD, i.e. B is lowered by omega b:
            // B = omega (bf - 1), with bf - 1 formed from rho - 1 (no cancellation).
            constexpr bool OF = Fmt<Q, S>::OFFSET;
            const T cf = T(1) - P.omega[0], cg = T(1) - P.omega[1], ck = T(1) - P.omega[2];
            const T Bf = P.omega[0] * (OF ? E.bf1 : E.bf), Rf = T(4.5) * P.omega[0] * E.rho,
                    Of = T(3) * P.omega[0] * E.rho;
            const T Bg = P.omega[1] * E.bg, Rg = T(4.5) * P.omega[1] * E.phi, Og = T(3) * P.omega[1] * E.phi;
            const T Bk = P.omega[2] * E.bk, Rk = T(4.5) * P.omega[2] * E.psi, Ok = T(3) * P.omega[2] * E.psi;
#pragma unroll
            for (int c = 0; c < 6; ++c) E.Gs[c] *= P.omega[0];
            T sf = T(0), sg = T(0), sk = T(0);  // sums of omega x_eq over moving links
            T qf = T(0), qg = T(0), qk = T(0);  // sums of the moving populations as stored
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const int o = opp<Q>(i);
                if (o < i) continue;
                const T w = T(Lat<Q>::w(i));
                const T e = E.eu(i);
                const T e2 = e * e;
                const T evf = w * (Bf + Rf * e2) + E.grad_term(i), odf = (w * Of) * e;
                const T evg = w * (Bg + Rg * e2), odg = (w * Og) * e;
                const T evk = w * (Bk + Rk * e2), odk = (w * Ok) * e;
                sf += T(2) * evf;
                sg += T(2) * evg;
                sk += T(2) * evk;
                const T v[6] = {cf * fv[i] + (evf + odf), cf * fv[o] + (evf - odf),
                                cg * gv[i] + (evg + odg), cg * gv[o] + (evg - odg),
                                ck * kv[i] + (evk + odk), ck * kv[o] + (evk - odk)};
                if constexpr (Fmt<Q, S>::PAIRED) {  // three lane words (all offset formats)
                    T q[6];  // the deviations as stored
                    Fmt<Q, S>::template st_fg_q<(HINT >= 1)>(out, i, v[0], v[2], q[0], q[2]);
                    Fmt<Q, S>::template st_fg_q<(HINT >= 1)>(out, o, v[1], v[3], q[1], q[3]);
                    Fmt<Q, S>::template st_kk_q<(HINT >= 1)>(out, i, v[4], v[5], q[4], q[5]);
                    qf += q[0] + q[1];
                    qg += q[2] + q[3];
                    qk += q[4] + q[5];
                } else {
                    st_(out, 0, i, v[0]);
                    st_(out, 0, o, v[1]);
                    st_(out, 1, i, v[2]);
                    st_(out, 1, o, v[3]);
                    st_(out, 2, i, v[4]);
                    st_(out, 2, o, v[5]);
                    if (OF) {
                        qf += Fmt<Q, S>::qdelta_d(i, v[0]) + Fmt<Q, S>::qdelta_d(o, v[1]);
                        qg += Fmt<Q, S>::qdelta_d(i, v[2]) + Fmt<Q, S>::qdelta_d(o, v[3]);
                        qk += Fmt<Q, S>::qdelta_d(i, v[4]) + Fmt<Q, S>::qdelta_d(o, v[5]);
                    }
                }
            }
            if (OF) {
                // rest = moment - moving populations as stored (deviations for f):
                // every node keeps its rho, phi, psi through the rounding of the
                // stored values (a rounding of the rest population alone)
                st_(out, 0, 0, rdc - qf);
                st_(out, 1, 0, E.phi - qg);
                st_(out, 2, 0, E.psi - qk);
            } else {
                // omega x_eq_0 = omega X - sum of omega x_eq over the moving links
                st_(out, 0, 0, cf * fv[0] + (P.omega[0] * E.rho - sf));
                st_(out, 1, 0, cg * gv[0] + (P.omega[1] * E.phi - sg));
                st_(out, 2, 0, ck * kv[0] + (P.omega[2] * E.psi - sk));
            }
        }
        jc[0] = jn[0];
        jc[1] = jn[1];
        jc[2] = jn[2];
        rdc = rdn;
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

template <int Q, typename S, int TX, int TY, bool ILP, bool EARLY, bool PF = false, int HINT = 0, bool CHK = false>
__global__ void __launch_bounds__(TX * TY, 512 / (TX * TY))  // 16 warps per SM
k_fused(MGeom g, const S* __restrict__ src, S* __restrict__ dst, Phys<typename Store<S>::T> P,
        double* __restrict__ partials) {
    fused_body<Q, S, TX, TY, ILP, EARLY, PF, HINT, 0, 1, CHK>(g, src, dst, P, partials, blockIdx.x);
}

// Variants of the periodic step with shared-memory staging of the pulled
// populations (STG values in the order STGO), at BPS blocks per SM.
template <int Q, typename S, int TX, int TY, int STG, int STGO, int BPS, bool ILP, bool PF, int HINT,
          bool CHK = false, int LDH = 0>
__global__ void __launch_bounds__(TX * TY, BPS)
k_fused_x(MGeom g, const S* __restrict__ src, S* __restrict__ dst, Phys<typename Store<S>::T> P,
          double* __restrict__ partials) {
    fused_body<Q, S, TX, TY, ILP, false, PF, HINT, STG, STGO, CHK, LDH>(g, src, dst, P, partials, blockIdx.x);
}

// ------------------------------------------------------ solid-aware variant

// Bit i (1 <= i < Q) of nbm[r]: the pull source r - e_i of node r is solid;
// bit 0: r itself is solid.  Built once per lattice.
template <int Q>
__global__ void k_nbmask(Geom g, const uint8_t* __restrict__ solid, uint32_t* __restrict__ nbm) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.N;
         r += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords(g, r, x, y, z);
        uint32_t m = solid[r] ? 1u : 0u;
#pragma unroll
        for (int i = 1; i < Q; ++i)
            if (solid[node(g, wrap(x - Lat<Q>::cx(i), g.nx), wrap(y - Lat<Q>::cy(i), g.ny),
                           wrap(z - Lat<Q>::cz(i), g.nz))])
                m |= 1u << i;
        nbm[r] = m;
    }
}

// One step with solid nodes, halfway bounce-back and wetting ghosts.  As
// k_fused, but the ghost value of a solid node needs the moments of its fluid
// neighbours, so each block keeps a two-node halo and works two planes ahead:
//   M(m+2): moments of plane m+2 over tile + 2-node halo (solid nodes: 0)
//   barrier
//   G(m+1): ghost values of the solid nodes of plane m+1 over tile + 1-node halo
//           (mean over fluid axis neighbours of X - G_X; with only diagonal
//           fluid neighbours, of X - sqrt(2) G_X)
//   barrier
//   C(m):   derivatives, equilibria, BGK and store for the fluid tile nodes.
// The moment and mask rings have five plane slots and the momentum ring four, so
// a fast warp writing plane m+2 never touches data a slow warp still reads.
template <int Q, typename S, int TX, int TY, bool CHK = false>
__device__ __forceinline__ void solid_body(const MGeom& g, const S* __restrict__ src, S* __restrict__ dst,
                                           const uint32_t* __restrict__ nbm,
                                           const Phys<typename Store<S>::T>& P, double* __restrict__ partials,
                                           const int bid) {
    using T = typename Store<S>::T;
    using A = Axes<Q>;
    constexpr int D = Lat<Q>::D;
    constexpr int H = 2;                  // halo width along a
    constexpr int HB = (D == 3) ? 2 : 0;  // halo width along b
    constexpr int HW = TX + 2 * H;
    constexpr int HH = TY + 2 * HB;
    constexpr int HN = HW * HH;
    constexpr int NT = TX * TY;
    constexpr int KS = (HN + NT - 1) / NT;  // region nodes per thread
    constexpr int R = 5;                    // plane slots of the rings
    static_assert(D == 3 || TY == 1, "2-D tiles are one row");
    static_assert(KS <= 3, "at most three region nodes per thread");

    __shared__ T sm[R][3][HN];       // effective rho, phi, psi (ghosts on solid nodes)
    __shared__ uint32_t sk[R][HN];   // neighbour masks
    __shared__ T sj[4][4][NT];       // j and summed f deviations of the tile

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
    const long long plane = (long long)g.NA * g.NB;

    // this thread's region nodes h = tid + k NT: in-plane node index, pull-source
    // byte offsets along a and rows along b
    int xc[KS][3], yb[KS][3], rin[KS];
#pragma unroll
    for (int k = 0; k < KS; ++k) {
        const int h = min(tid + k * NT, HN - 1);
        const int hx = h % HW, hy = h / HW;
        const int aa = modp(A0 + hx - H, g.NA);
        const int bb = (D == 3) ? modp(B0 + hy - HB, g.NB) : 0;
        const int xs[3] = {wrap1(aa - 1, g.NA), aa, wrap1(aa + 1, g.NA)};
#pragma unroll
        for (int c = 0; c < 3; ++c) xc[k][c] = (xs[c] >> 5) * (int)Fmt<Q, S>::CHUNK + (xs[c] & 31) * Fmt<Q, S>::ESZ;
        yb[k][0] = (D == 3) ? wrap1(bb - 1, g.NB) : 0;
        yb[k][1] = bb;
        yb[k][2] = (D == 3) ? wrap1(bb + 1, g.NB) : 0;
        rin[k] = aa + g.NA * bb;
    }
    // the thread's own tile node (phase C): byte offsets of a-1, a, a+1, rows b-1, b, b+1
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
    const unsigned char* srcb = reinterpret_cast<const unsigned char*>(src);
    auto row_ptr = [&](int k, const int (&zr)[3], int cb, int cm) -> const unsigned char* {
        return srcb + ((long long)zr[1 - cm] * g.NB + yb[k][1 - cb]) * g.rowstride;
    };
    auto own_row = [&](const int (&zr)[3], int cb, int cm) -> const unsigned char* {
        return srcb + ((long long)zr[1 - cm] * g.NB + yo[1 - cb]) * g.rowstride;
    };

    // M: moments of plane m (node k's pulled populations, bounce-back at solids)
    auto moments_plane = [&](int m) {
        const int mm = modp(m, g.NM), slot = modp(m, R), js = modp(m, 4);
        const int zr[3] = {wrap1(mm - 1, g.NM), mm, wrap1(mm + 1, g.NM)};
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const int h = tid + k * NT;
            if (h >= HN) break;
            const uint32_t mk = nbm[chk_index<CHK>(g, (long long)mm * plane + rin[k], plane * g.NM, 5)];
            T rd = T(0), ja = T(0), jb = T(0), jm = T(0), phi = T(0), psi = T(0);
            if (!(mk & 1u)) {
                const unsigned char* own = chk_node<Q, S, CHK>(g, srcb, row_ptr(k, zr, 0, 0) + xc[k][1], 2);
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    // pull source, or this node's opposite run when the source is solid:
                    // one pointer select, then loads at the run offsets of direction i
                    // (pointer selects per set: f and g of a direction move together, k apart)
                    const unsigned char* p =
                        chk_node<Q, S, CHK>(g, srcb, row_ptr(k, zr, A::cb(i), A::cm(i)) + xc[k][1 - A::ca(i)], 1);
                    const bool bb = i > 0 && ((mk >> i) & 1u);
                    const unsigned char* pfg = bb ? own + (Fmt<Q, S>::off(0, opp<Q>(i)) - Fmt<Q, S>::off(0, i)) : p;
                    const unsigned char* pk = bb ? own + (Fmt<Q, S>::off(2, opp<Q>(i)) - Fmt<Q, S>::off(2, i)) : p;
                    T f, gv;
                    if (i > 0) Fmt<Q, S>::ld_fg(pfg, i, f, gv);
                    else f = Fmt<Q, S>::ld_delta(p, 0, 0), gv = Fmt<Q, S>::ld_delta(p, 1, 0);
                    rd += f;
                    if (A::ca(i)) ja += T(A::ca(i)) * f;
                    if (A::cb(i)) jb += T(A::cb(i)) * f;
                    if (A::cm(i)) jm += T(A::cm(i)) * f;
                    phi += gv;
                    psi += Fmt<Q, S>::ld_delta(pk, 2, i);
                }
            }
            const T rho = (mk & 1u) ? T(0) : (Fmt<Q, S>::OFFSET ? T(1) + rd : rd);
            sm[slot][0][h] = rho;
            sm[slot][1][h] = phi;
            sm[slot][2][h] = psi;
            sk[slot][h] = mk;
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

    // G: ghost values of the solid nodes of plane q within the one-node halo
    auto ghosts_plane = [&](int q) {
        const int slot = modp(q, R);
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const int h = tid + k * NT;
            if (h >= HN) break;
            const int hx = h % HW, hy = h / HW;
            if (hx < 1 || hx > HW - 2 || (D == 3 && (hy < 1 || hy > HH - 2))) continue;
            const uint32_t mk = sk[slot][h];
            if (!(mk & 1u)) continue;
            T acc[3] = {T(0), T(0), T(0)};
            int n = 0;
#pragma unroll
            for (int i = 1; i <= Lat<Q>::NAXIS; ++i) {  // neighbour s + e_i is fluid?
                if ((mk >> opp<Q>(i)) & 1u) continue;
                const int sn = modp(q + A::cm(i), R);
                const int hn = (int)chk_index<CHK>(g, h + A::cb(i) * HW + A::ca(i), HN, 4);
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[c] += sm[sn][c][hn] - P.Gw[c];
                ++n;
            }
            if (n == 0) {
                const T r2 = T(1.4142135623730951);
#pragma unroll
                for (int i = Lat<Q>::NAXIS + 1; i < Q; ++i) {
                    if ((mk >> opp<Q>(i)) & 1u) continue;
                    const int sn = modp(q + A::cm(i), R);
                    const int hn = (int)chk_index<CHK>(g, h + A::cb(i) * HW + A::ca(i), HN, 4);
#pragma unroll
                    for (int c = 0; c < 3; ++c) acc[c] += sm[sn][c][hn] - r2 * P.Gw[c];
                    ++n;
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) sm[slot][c][h] = n > 0 ? acc[c] / T(n) : T(0);
        }
    };

    constexpr bool PAIR = Fmt<Q, S>::OFFSET && !(Q == 19 && sizeof(S) == 4);
    constexpr bool HL = sizeof(S) == 4;  // evict-first hints in the collision
    MassSum<T, PAIR> msum;

    moments_plane(M0 - 2);
    moments_plane(M0 - 1);
    moments_plane(M0);
    moments_plane(M0 + 1);
    __syncthreads();
    ghosts_plane(M0 - 1);
    ghosts_plane(M0);
    __syncthreads();

    const int c0 = (ty + HB) * HW + tx + H;  // this thread's tile node in the region
    for (int m = M0; m < M1; ++m) {
        moments_plane(m + 2);
        __syncthreads();
        ghosts_plane(m + 1);
        __syncthreads();
        const int s0 = modp(m, R);
        const uint32_t mk = sk[s0][c0];
        if (!active || (mk & 1u)) continue;

        // ---- derivatives from the ring (ghost values on solid neighbours)
        T X0[3], gA[3], gB[3], gM[3], lp[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            X0[c] = sm[s0][c][c0];
            gA[c] = gB[c] = gM[c] = lp[c] = T(0);
        }
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if (opp<Q>(i) < i) continue;
            const int sp = modp(m + A::cm(i), R), sn = modp(m - A::cm(i), R);
            const int cp = (int)chk_index<CHK>(g, c0 + A::cb(i) * HW + A::ca(i), HN, 4);
            const int cn = (int)chk_index<CHK>(g, c0 - A::cb(i) * HW - A::ca(i), HN, 4);
            const T w = T(Lat<Q>::w(i));
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T xpv = sm[sp][c][cp], xnv = sm[sn][c][cn];
                const T d = w * (xpv - xnv);
                if (A::ca(i)) gA[c] += T(A::ca(i)) * d;
                if (A::cb(i)) gB[c] += T(A::cb(i)) * d;
                if (A::cm(i)) gM[c] += T(A::cm(i)) * d;
                lp[c] += w * (xpv + xnv);
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
        const int t = ty * TX + tx, js = modp(m, 4);
        const T jA = sj[js][0][t], jB = sj[js][1][t], jM = sj[js][2][t], rdc = sj[js][3][t];
        NodeEq<Q, T> E;
        if (D == 3) E.setup(P, X0[0], jA, jB, jM, X0[1], X0[2], grad, lap);
        else E.setup(P, X0[0], jA, jM, T(0), X0[1], X0[2], grad, lap);
        if constexpr (PAIR) msum.add(rdc, X0[1], X0[2]);
        else msum.add(rho_total<Q, S>(rdc), X0[1], X0[2]);

        // ---- pulled populations (bounce-back at solid sources)
        const int zr[3] = {wrap1(m - 1, g.NM), m, wrap1(m + 1, g.NM)};
        const unsigned char* own = chk_node<Q, S, CHK>(g, srcb, own_row(zr, 0, 0) + xo[1], 2);
        T fv[Q], gv[Q], kv[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const unsigned char* p = chk_node<Q, S, CHK>(g, srcb, own_row(zr, A::cb(i), A::cm(i)) + xo[1 - A::ca(i)], 1);
            const bool bb = i > 0 && ((mk >> i) & 1u);
            const unsigned char* pfg = bb ? own + (Fmt<Q, S>::off(0, opp<Q>(i)) - Fmt<Q, S>::off(0, i)) : p;
            const unsigned char* pk = bb ? own + (Fmt<Q, S>::off(2, opp<Q>(i)) - Fmt<Q, S>::off(2, i)) : p;
            // the collision is the last reader of these lines: evict-first loads
            // (FP32 storage; measured slower for the 16-bit formats)
            if (i > 0) {
                T df, dg;
                Fmt<Q, S>::template ld_fg<HL>(pfg, i, df, dg);
                fv[i] = Fmt<Q, S>::unbias(0, i, df);
                gv[i] = dg;
            } else {
                fv[i] = HL ? Fmt<Q, S>::ld_last(p, 0, 0) : Fmt<Q, S>::ld(p, 0, 0);
                gv[i] = HL ? Fmt<Q, S>::ld_last(p, 1, 0) : Fmt<Q, S>::ld(p, 1, 0);
            }
            kv[i] = HL ? Fmt<Q, S>::ld_last(pk, 2, i) : Fmt<Q, S>::ld(pk, 2, i);
        }

        // ---- collide + store (same arithmetic as k_fused)
        unsigned char* out = chk_node<Q, S, CHK>(
            g, reinterpret_cast<unsigned char*>(dst),
            reinterpret_cast<unsigned char*>(dst) + ((long long)m * g.NB + yo[1]) * g.rowstride + xo[1], 3);
        const T cf = T(1) - P.omega[0], cg = T(1) - P.omega[1], ck = T(1) - P.omega[2];
        const T Bf = P.omega[0] * E.bf, Rf = T(4.5) * P.omega[0] * E.rho, Of = T(3) * P.omega[0] * E.rho;
        const T Bg = P.omega[1] * E.bg, Rg = T(4.5) * P.omega[1] * E.phi, Og = T(3) * P.omega[1] * E.phi;
        const T Bk = P.omega[2] * E.bk, Rk = T(4.5) * P.omega[2] * E.psi, Ok = T(3) * P.omega[2] * E.psi;
#pragma unroll
        for (int c = 0; c < 6; ++c) E.Gs[c] *= P.omega[0];
        T sf = T(0), sg = T(0), sk2 = T(0), qf = T(0), qg = T(0), qk = T(0);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int o = opp<Q>(i);
            if (o < i) continue;
            const T w = T(Lat<Q>::w(i));
            const T e = E.eu(i);
            const T e2 = e * e;
            const T evf = w * (Bf + Rf * e2) + E.grad_term(i), odf = (w * Of) * e;
            const T evg = w * (Bg + Rg * e2), odg = (w * Og) * e;
            const T evk = w * (Bk + Rk * e2), odk = (w * Ok) * e;
            sf += T(2) * evf;
            sg += T(2) * evg;
            sk2 += T(2) * evk;
            const T v[6] = {cf * fv[i] + (evf + odf), cf * fv[o] + (evf - odf),
                            cg * gv[i] + (evg + odg), cg * gv[o] + (evg - odg),
                            ck * kv[i] + (evk + odk), ck * kv[o] + (evk - odk)};
            // streamed out (evict-first, FP32): read only by the next step
            Fmt<Q, S>::template st_fg<HL>(out, i, Fmt<Q, S>::dev(0, i, v[0]), v[2]);
            Fmt<Q, S>::template st_fg<HL>(out, o, Fmt<Q, S>::dev(0, o, v[1]), v[3]);
            Fmt<Q, S>::template st_kk<HL>(out, i, v[4], v[5]);
            if (Fmt<Q, S>::OFFSET) {
                qf += Fmt<Q, S>::qdelta(0, i, v[0]) + Fmt<Q, S>::qdelta(0, o, v[1]);
                qg += Fmt<Q, S>::qdelta(1, i, v[2]) + Fmt<Q, S>::qdelta(1, o, v[3]);
                qk += Fmt<Q, S>::qdelta(2, i, v[4]) + Fmt<Q, S>::qdelta(2, o, v[5]);
            }
        }
        auto st_rest = [&](int s_, T d) {
            if (HL) Fmt<Q, S>::st_stream_delta(out, s_, 0, d);
            else Fmt<Q, S>::st_delta(out, s_, 0, d);
        };
        if (Fmt<Q, S>::OFFSET) {
            st_rest(0, rdc - qf);
            st_rest(1, E.phi - qg);
            st_rest(2, E.psi - qk);
        } else {
            st_rest(0, Fmt<Q, S>::dev(0, 0, cf * fv[0] + (P.omega[0] * E.rho - sf)));
            st_rest(1, cg * gv[0] + (P.omega[1] * E.phi - sg));
            st_rest(2, ck * kv[0] + (P.omega[2] * E.psi - sk2));
        }
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

template <int Q, typename S, int TX, int TY, bool CHK = false>
__global__ void __launch_bounds__(TX * TY, 512 / (TX * TY))
k_fused_solid(MGeom g, const S* __restrict__ src, S* __restrict__ dst, const uint32_t* __restrict__ nbm,
              Phys<typename Store<S>::T> P, double* __restrict__ partials) {
    solid_body<Q, S, TX, TY, CHK>(g, src, dst, nbm, P, partials, blockIdx.x);
}

// ------------------------------------------------------------- batches

// One member of a batched step: its geometry, buffers for this step's parity,
// neighbour mask (solid lattices), physics, partial sums and first block.
template <typename T>
struct SimDesc {
    MGeom g;
    const void* src;
    void* dst;
    const uint32_t* nbm;
    Phys<T> P;
    double* partials;
    double* step_mass;
    int* flag;
    int block0;  // first block of this member in the batched grid
    int nblocks;
};

// block -> member: the last descriptor whose block0 <= blockIdx.x; the member's
// descriptor is copied to shared memory for the body to read
template <typename T>
__device__ __forceinline__ const SimDesc<T>& batch_member(const SimDesc<T>* __restrict__ d, int nsims,
                                                          SimDesc<T>& sh) {
    if (threadIdx.x == 0) {
        int lo = 0, hi = nsims - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (d[mid].block0 <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        sh = d[lo];
    }
    __syncthreads();
    return sh;
}

template <int Q, typename S, int TX, int TY, bool PF, int HINT>
__global__ void __launch_bounds__(TX * TY, 512 / (TX * TY))
k_fused_batch(const SimDesc<typename Store<S>::T>* __restrict__ d, int nsims) {
    __shared__ SimDesc<typename Store<S>::T> sh;
    const SimDesc<typename Store<S>::T>& m = batch_member(d, nsims, sh);
    fused_body<Q, S, TX, TY, false, false, PF, HINT>(m.g, static_cast<const S*>(m.src), static_cast<S*>(m.dst),
                                                     m.P, m.partials, (int)blockIdx.x - m.block0);
}

template <int Q, typename S, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, 512 / (TX * TY))
k_fused_solid_batch(const SimDesc<typename Store<S>::T>* __restrict__ d, int nsims) {
    __shared__ SimDesc<typename Store<S>::T> sh;
    const SimDesc<typename Store<S>::T>& m = batch_member(d, nsims, sh);
    solid_body<Q, S, TX, TY>(m.g, static_cast<const S*>(m.src), static_cast<S*>(m.dst), m.nbm, m.P,
                             m.partials, (int)blockIdx.x - m.block0);
}

// FP64 totals of every member: block i sums member i's partials in a fixed order
template <typename T>
__global__ void k_mass_final_batch(const SimDesc<T>* __restrict__ d) {
    const SimDesc<T>& m = d[blockIdx.x];
    double a = 0.0, b = 0.0, c = 0.0;
    for (int k = threadIdx.x; k < m.nblocks; k += blockDim.x) {
        a += m.partials[3 * k];
        b += m.partials[3 * k + 1];
        c += m.partials[3 * k + 2];
    }
    block_sum3(a, b, c);
    if (threadIdx.x == 0) {
        m.step_mass[0] = a;
        m.step_mass[1] = b;
        m.step_mass[2] = c;
        if (!(isfinite(a) && isfinite(b) && isfinite(c))) *m.flag = 1;
    }
}

// ------------------------------------------------------------ host side

// grid of a grid-stride kernel of 256 threads over n items: at most 8 blocks
// per SM (results do not depend on it)
inline int grid_of(long long n, int sms) {
    const long long b = (n + 255) / 256, cap = 8LL * (sms < 1 ? 1 : sms);
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <int Q>
struct FusedCfg {
    int TX, TY, MC;
    int mode;
    int shape;  // resolved D3Q19 shape (4..7: 32x4 kernels with staging)
};

// d.tile = shape | mode << 4 | chunk << 8: shape 0 = default (D3Q19 shape 7,
// D2Q9 shape 5); D3Q19 1 = 32x8, 2 = 64x4, 3 = 32x4, 4..7 = 32x4 with the pulled
// populations of a thread's node staged in shared memory for the collision
// (4: the 19 f values; 5: lane-shifted values first, 28 for FP32, 19 with the
// per-warp prefetch for 16-bit storage; 6: 19 lane-shifted values; 7: as 5 in
// the order of the paired lane words, the k values first, then the
// lane-shifted (f, g) pairs, so that the collision reloads whole words); D2Q9
// shape 0 = 5: 128-node rows with all 27 values staged, 1 = 128, 2 = 256, 3 =
// 64, 4 = 128 with the 18 lane-shifted values staged.  mode (shapes 1..3) bit 0: interleaved border
// loads; bit 1: early phase-C loads; bit 2: per-warp L2 prefetch three planes
// ahead; 8 / 9: evict-first stores / stores and collision loads (12, 13 with
// the prefetch).  mode 0 is the default for the shape and format (D3Q19 32x4:
// 8 for FP32, 12 for 16-bit storage; other D3Q19: 1; D2Q9: 13); 6 selects the
// plain loop.  chunk = planes per block (0 = chosen from the lattice size).
template <int Q>
inline FusedCfg<Q> fused_cfg(const tlbm_host::DevState& d) {
    const bool dbl = d.prec == 0;  // double storage: one default shape only
    const int tile = d.checked ? 0 : d.tile;  // the checked kernels use the default tile
    const int variant = dbl ? 0 : (tile & 15);
    int mc = tile >> 8;
    FusedCfg<Q> c{};
    if (d.coupling) {
        // forcing coupling (k_guo_fused): the solid-aware kernel's tiles (two-node halo)
        c.TX = Q == 19 ? (dbl ? 16 : 32) : 128;
        c.TY = Q == 19 ? 4 : 1;
    } else if (d.solid) {
        // solid-aware kernel: a fixed tile per lattice (D3Q19 in double: 16x4 keeps
        // its five-plane rings under the 48 KB static shared-memory limit)
        c.TX = Q == 19 ? (dbl ? 16 : 32) : (dbl ? 128 : (variant == 2 ? 256 : (variant == 3 ? 64 : 128)));
        c.TY = Q == 19 ? 4 : 1;
    } else if (Q == 19 && dbl) {
        c.TX = 16;  // double storage: a smaller tile keeps the static shared ring small
        c.TY = 8;
    } else if (Q == 19) {
        const int v = variant == 0 ? 7 : variant;  // 32x4 with pair-aware staging measured fastest on 256^3
        c.TX = v == 2 ? 64 : 32;
        c.TY = v == 1 ? 8 : 4;
        c.shape = v;
    } else {
        const int v = variant == 0 ? 5 : variant;  // 128-node rows with staging measured fastest
        c.TX = v == 2 ? 256 : (v == 3 ? 64 : 128);
        c.TY = 1;
        c.shape = v;
    }
    c.mode = dbl ? 0 : ((tile >> 4) & 15);
    // defaults measured on GB300: D3Q19 32x4 with evict-first stores, plus a
    // per-warp L2 prefetch for the 16-bit formats (a plane of FP32 populations
    // is too large for the prefetch to stay in L2); 64x4 and 32x8 interleaved
    // border loads; D2Q9 prefetch, evict-first stores and collision loads
    if (c.mode == 0)
        c.mode = (Q == 19) ? (c.TX == 32 && c.TY == 4 ? (d.prec >= 2 ? 12 : 8) : 1) : 13;
    const int NA = d.nx;
    const int NB = (Q == 19) ? d.ny : 1;
    const int NM = (Q == 19) ? d.nz : d.ny;
    if (mc <= 0) {
        // enough blocks to fill every SM of the device a few times over
        const long long cols = (long long)((NA + c.TX - 1) / c.TX) * ((NB + c.TY - 1) / c.TY);
        mc = (Q == 19) ? 16 : 64;
        while (mc > 4 && cols * ((NM + mc - 1) / mc) < 4LL * d.sms) mc >>= 1;
    }
    c.MC = mc < 1 ? 1 : (mc > NM ? NM : mc);
    return c;
}

template <int Q, typename S>
inline bool fused_supported(const tlbm_host::DevState& d) {
    return d.solid == nullptr || d.nbm != nullptr;
}

template <int Q, typename S>
inline int fused_launches(const tlbm_host::DevState&) {
    return 1;
}

template <int Q, typename S>
inline MGeom mgeom(const tlbm_host::DevState& d, const FusedCfg<Q>& c) {
    MGeom g;
    g.NA = d.nx;
    g.NB = (Q == 19) ? d.ny : 1;
    g.NM = (Q == 19) ? d.nz : d.ny;
    g.rowstride = (long long)d.ncx * Fmt<Q, S>::CHUNK;
    g.NC = (g.NM + c.MC - 1) / c.MC;  // chunks of MC planes or one fewer (balanced)
    g.bytes = d.pop_bytes;
    g.check = d.check;
    g.tilesA = (g.NA + c.TX - 1) / c.TX;
    g.tilesB = (g.NB + c.TY - 1) / c.TY;
    return g;
}

template <int Q, typename S>
inline long long fused_blocks(const tlbm_host::DevState& d) {
    const FusedCfg<Q> c = fused_cfg<Q>(d);
    const MGeom g = mgeom<Q, S>(d, c);
    return (long long)g.tilesA * g.tilesB * g.NC;
}

// number of partial sums the last step wrote (for k_mass_final)
template <int Q, typename S>
inline int fused_partials(const tlbm_host::DevState& d, int kind) {
    return kind == tlbm_host::KIND_FUSED ? (int)fused_blocks<Q, S>(d) : kMassBlocks;
}

// Launch of a kernel with STG staged values per thread of 128 (dynamic shared
// memory), with the smallest shared-memory carveout that still holds four
// blocks per SM, so that the rest of the SM's 256 KB stays L1 (which holds the
// kernel's loads in flight).
template <typename K, typename... Args>
inline cudaError_t launch_staged_t(K kern, int stg, int threads, int bps, long long nb, cudaStream_t st,
                                   Args... args) {
    const int dyn = stg * 2 * threads * (int)sizeof(float);
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return e;
    const long long need = (long long)bps * ((long long)fa.sharedSizeBytes + dyn + 1024);
    const int pct = (int)((need * 100 + 233471) / 233472);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct > 100 ? 100 : pct);
    if (e != cudaSuccess) return e;
    kern<<<(int)nb, threads, dyn, st>>>(args...);
    return cudaSuccess;
}
template <typename K, typename... Args>
inline cudaError_t launch_staged(K kern, int stg, long long nb, cudaStream_t st, Args... args) {
    return launch_staged_t(kern, stg, 128, 4, nb, st, args...);
}

template <int Q, typename S>
inline cudaError_t fused_step(tlbm_host::DevState& d, const Phys<typename Store<S>::T>& P, cudaStream_t st) {
    const FusedCfg<Q> c = fused_cfg<Q>(d);
    const MGeom g = mgeom<Q, S>(d, c);
    const long long nb = (long long)g.tilesA * g.tilesB * g.NC;
    if (nb > 0x7fffffffLL || nb > d.partials_cap) return cudaErrorInvalidConfiguration;
    const S* src = static_cast<const S*>(d.pop[d.cur]);
    S* dst = static_cast<S*>(d.pop[1 - d.cur]);
    if (d.solid && !d.nbm_ready) {
        const Geom gg{d.nx, d.ny, d.nz, d.N, d.Np, d.ncx};
        k_nbmask<Q><<<grid_of(d.N, d.sms), 256, 0, st>>>(gg, d.solid, d.nbm);
        d.nbm_ready = 1;
    }
    if (d.checked) {
        // bounds-checked kernels of the default FP32 tiles (recording, never trapping)
        if constexpr (sizeof(S) == 4) {
            if (!d.check) return cudaErrorInvalidValue;
            if (d.solid) {
                if constexpr (Q == 19) k_fused_solid<Q, S, 32, 4, true><<<(int)nb, 128, 0, st>>>(g, src, dst, d.nbm, P, d.partials);
                else k_fused_solid<Q, S, 128, 1, true><<<(int)nb, 128, 0, st>>>(g, src, dst, d.nbm, P, d.partials);
            } else {
                if constexpr (Q == 19) {
                    const cudaError_t e = launch_staged(k_fused_x<Q, S, 32, 4, 28, 2, 4, false, false, 1, true>, 28, nb,
                                                        st, g, src, dst, P, d.partials);
                    if (e != cudaSuccess) return e;
                } else {
                    const cudaError_t e = launch_staged(k_fused_x<Q, S, 128, 1, 27, 0, 4, false, true, 2, true>, 27, nb,
                                                        st, g, src, dst, P, d.partials);
                    if (e != cudaSuccess) return e;
                }
            }
            return cudaGetLastError();
        } else {
            return cudaErrorNotSupported;
        }
    }
    if (d.solid) {
        auto gos = [&](auto kern, int threads) {
            kern<<<(int)nb, threads, 0, st>>>(g, src, dst, d.nbm, P, d.partials);
        };
        if constexpr (Q == 19) {
            if constexpr (sizeof(S) == 8) gos(k_fused_solid<Q, S, 16, 4>, 64);
            else gos(k_fused_solid<Q, S, 32, 4>, 128);
        } else {
            if (c.TX == 256) gos(k_fused_solid<Q, S, 256, 1>, 256);
            else if (c.TX == 64) gos(k_fused_solid<Q, S, 64, 1>, 64);
            else gos(k_fused_solid<Q, S, 128, 1>, 128);
        }
        return cudaGetLastError();
    }
    auto go = [&](auto kern, int threads) { kern<<<(int)nb, threads, 0, st>>>(g, src, dst, P, d.partials); };
    if constexpr (sizeof(S) == 8) {
        // double storage is the parity path: one tile shape per lattice
        if constexpr (Q == 19) go(k_fused<Q, S, 16, 8, false, false>, 128);
        else go(k_fused<Q, S, 128, 1, false, false>, 128);
    } else if constexpr (Q == 19) {
        if constexpr (sizeof(S) <= 4) {
            if (c.shape >= 4) {
                // 32x4 kernels with shared-memory staging of the pulled populations:
                // 4 the 19 f values; 5 the lane-shifted values first, 28 of them for
                // FP32, 19 with the per-warp L2 prefetch for the 16-bit formats; 6
                // 19 lane-shifted values (no prefetch); 7 (default) as 5 in the
                // paired-word order (k values, then lane-shifted (f, g) pairs)
                cudaError_t e;
                if constexpr (sizeof(S) == 2) {
                    switch (c.shape) {
                        case 4: e = launch_staged(k_fused_x<Q, S, 32, 4, 19, 1, 4, false, true, 1>, 19, nb, st, g, src, dst, P, d.partials); break;
                        case 6: e = launch_staged(k_fused_x<Q, S, 32, 4, 19, 0, 4, false, false, 1>, 19, nb, st, g, src, dst, P, d.partials); break;
                        case 5: e = launch_staged(k_fused_x<Q, S, 32, 4, 19, 0, 4, false, true, 1>, 19, nb, st, g, src, dst, P, d.partials); break;
                        default: e = launch_staged(k_fused_x<Q, S, 32, 4, 19, 2, 4, false, true, 1>, 19, nb, st, g, src, dst, P, d.partials);
                    }
                } else {
                    switch (c.shape) {
                        case 4: e = launch_staged(k_fused_x<Q, S, 32, 4, 19, 1, 4, false, false, 1>, 19, nb, st, g, src, dst, P, d.partials); break;
                        case 6: e = launch_staged(k_fused_x<Q, S, 32, 4, 19, 0, 4, false, false, 1>, 19, nb, st, g, src, dst, P, d.partials); break;
                        case 5: e = launch_staged(k_fused_x<Q, S, 32, 4, 28, 0, 4, false, false, 1>, 28, nb, st, g, src, dst, P, d.partials); break;
                        default: e = launch_staged(k_fused_x<Q, S, 32, 4, 28, 2, 4, false, false, 1>, 28, nb, st, g, src, dst, P, d.partials);
                    }
                }
                return e != cudaSuccess ? e : cudaGetLastError();
            }
        }
        if (c.TX == 64) {
            switch (c.mode) {
                case 2: go(k_fused<Q, S, 64, 4, false, true>, 256); break;
                case 4: go(k_fused<Q, S, 64, 4, false, false, true>, 256); break;
                case 5: go(k_fused<Q, S, 64, 4, true, false, true>, 256); break;
                case 6: go(k_fused<Q, S, 64, 4, false, false>, 256); break;
                default: go(k_fused<Q, S, 64, 4, true, false>, 256);
            }
        } else if (c.TY == 4) {
            switch (c.mode) {
                case 1: go(k_fused<Q, S, 32, 4, true, false>, 128); break;
                case 4: go(k_fused<Q, S, 32, 4, false, false, true>, 128); break;
                case 8: go(k_fused<Q, S, 32, 4, false, false, false, 1>, 128); break;
                case 9: go(k_fused<Q, S, 32, 4, false, false, false, 2>, 128); break;
                case 12: go(k_fused<Q, S, 32, 4, false, false, true, 1>, 128); break;
                case 13: go(k_fused<Q, S, 32, 4, false, false, true, 2>, 128); break;
                default: go(k_fused<Q, S, 32, 4, false, false>, 128);
            }
        } else {
            if (c.mode == 6) go(k_fused<Q, S, 32, 8, false, false>, 256);
            else go(k_fused<Q, S, 32, 8, true, false>, 256);
        }
    } else {
        if (c.shape >= 4 && !d.solid) {
            // 128-node rows with staging: 4 the 18 lane-shifted values, 5 (default)
            // all 27, with the per-warp prefetch and evict-first stores and
            // collision loads
            const cudaError_t e =
                c.shape == 4 ? launch_staged(k_fused_x<Q, S, 128, 1, 18, 0, 4, false, true, 2>, 18, nb, st, g, src, dst, P, d.partials)
                             : launch_staged(k_fused_x<Q, S, 128, 1, 27, 0, 4, false, true, 2>, 27, nb, st, g, src, dst, P, d.partials);
            return e != cudaSuccess ? e : cudaGetLastError();
        }
        if (c.TX == 256) {
            switch (c.mode) {
                case 1: go(k_fused<Q, S, 256, 1, true, false>, 256); break;
                case 2: go(k_fused<Q, S, 256, 1, false, true>, 256); break;
                case 3: go(k_fused<Q, S, 256, 1, true, true>, 256); break;
                default: go(k_fused<Q, S, 256, 1, false, false>, 256);
            }
        } else if (c.TX == 64) {
            go(k_fused<Q, S, 64, 1, false, false>, 64);
        } else if (c.mode == 4) {
            go(k_fused<Q, S, 128, 1, false, false, true>, 128);
        } else if (c.mode == 12) {
            go(k_fused<Q, S, 128, 1, false, false, true, 1>, 128);
        } else if (c.mode == 13) {
            go(k_fused<Q, S, 128, 1, false, false, true, 2>, 128);
        } else {
            go(k_fused<Q, S, 128, 1, false, false>, 128);  // plain loop
        }
    }
    return cudaGetLastError();
}

// ---- batches: every member uses the batch's tile; descriptors for both parities

template <int Q, typename S>
inline cudaError_t batch_build(tlbm_host::BatchState& b, cudaStream_t st) {
    using T = typename Store<S>::T;
    const int n = b.count;
    if (n < 1) return cudaErrorInvalidValue;
    const bool solid = b.sims[0]->solid != nullptr;
    std::vector<SimDesc<T>> h(2 * (size_t)n);
    long long block0 = 0;
    for (int k = 0; k < n; ++k) {
        tlbm_host::DevState& d = *b.sims[k];
        if ((d.solid != nullptr) != solid || d.cur != b.sims[0]->cur) return cudaErrorInvalidValue;
        if (solid && !d.nbm_ready) {
            const Geom gg{d.nx, d.ny, d.nz, d.N, d.Np, d.ncx};
            k_nbmask<Q><<<grid_of(d.N, d.sms), 256, 0, st>>>(gg, d.solid, d.nbm);
            d.nbm_ready = 1;
        }
        tlbm_host::DevState dd = d;
        dd.tile = b.tile;
        const FusedCfg<Q> c = fused_cfg<Q>(dd);
        // shapes with a batched kernel (batch_step): every solid shape; periodic
        // D3Q19 32x4 (16x8 in double), periodic D2Q9 128
        const bool shape_ok = solid || (Q == 19 ? (sizeof(S) == 8 ? (c.TX == 16 && c.TY == 8) : (c.TX == 32 && c.TY == 4))
                                                : c.TX == 128);
        if (!shape_ok) return cudaErrorInvalidConfiguration;
        const MGeom g = mgeom<Q, S>(dd, c);
        const long long nb = (long long)g.tilesA * g.tilesB * g.NC;
        if (nb > d.partials_cap) return cudaErrorInvalidConfiguration;
        for (int par = 0; par < 2; ++par) {
            SimDesc<T>& e = h[(size_t)par * n + k];
            e.g = g;
            e.src = d.pop[par];
            e.dst = d.pop[1 - par];
            e.nbm = d.nbm;
            e.P = to_phys<T>(d.phys);
            e.partials = d.partials;
            e.step_mass = d.step_mass;
            e.flag = d.flag;
            e.block0 = (int)block0;
            e.nblocks = (int)nb;
        }
        block0 += nb;
    }
    if (block0 > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    b.blocks = block0;
    cudaError_t e = cudaSuccess;
    if (!b.desc) e = cudaMalloc(&b.desc, sizeof(SimDesc<T>) * 2 * (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.desc, h.data(), sizeof(SimDesc<T>) * 2 * (size_t)n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) b.built = 1;
    return e;
}

template <int Q, typename S>
inline cudaError_t batch_step(tlbm_host::BatchState& b, cudaStream_t st, cudaEvent_t ev0 = nullptr,
                              cudaEvent_t ev1 = nullptr) {
    using T = typename Store<S>::T;
    const int n = b.count;
    const int par = b.sims[0]->cur;
    const SimDesc<T>* d = static_cast<const SimDesc<T>*>(b.desc) + (size_t)par * n;
    tlbm_host::DevState probe = *b.sims[0];
    probe.tile = b.tile;
    const FusedCfg<Q> c = fused_cfg<Q>(probe);
    const int nb = (int)b.blocks;
    if (ev0) cudaEventRecord(ev0, st);
    if (probe.solid) {
        if constexpr (Q == 19) {
            if constexpr (sizeof(S) == 8) k_fused_solid_batch<Q, S, 16, 4><<<nb, 64, 0, st>>>(d, n);
            else k_fused_solid_batch<Q, S, 32, 4><<<nb, 128, 0, st>>>(d, n);
        } else {
            if (c.TX == 256) k_fused_solid_batch<Q, S, 256, 1><<<nb, 256, 0, st>>>(d, n);
            else if (c.TX == 64) k_fused_solid_batch<Q, S, 64, 1><<<nb, 64, 0, st>>>(d, n);
            else k_fused_solid_batch<Q, S, 128, 1><<<nb, 128, 0, st>>>(d, n);
        }
    } else {
        if constexpr (Q == 19) {
            if constexpr (sizeof(S) == 8) k_fused_batch<Q, S, 16, 8, false, 0><<<nb, 128, 0, st>>>(d, n);
            else if constexpr (sizeof(S) == 2) k_fused_batch<Q, S, 32, 4, true, 1><<<nb, 128, 0, st>>>(d, n);
            else k_fused_batch<Q, S, 32, 4, false, 1><<<nb, 128, 0, st>>>(d, n);
        } else {
            k_fused_batch<Q, S, 128, 1, true, 2><<<nb, 128, 0, st>>>(d, n);
        }
    }
    if (ev1) cudaEventRecord(ev1, st);
    k_mass_final_batch<T><<<n, kThreads, 0, st>>>(d);
    for (int k = 0; k < n; ++k) b.sims[k]->cur ^= 1;
    return cudaGetLastError();
}

}  // namespace tlbm_dev
