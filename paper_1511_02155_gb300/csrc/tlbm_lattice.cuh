// tlbm_lattice.cuh -- velocity sets, weights, gradient-term tensors, storage
// formats and the per-node physics of the ternary free-energy LB step
// (Semprebon, Krueger, Kusumaatmaja, arXiv:1511.02155), for the GPU path.
//
// Everything here is compile-time: velocity components and weights are
// constexpr functions that fold to immediates once the direction loops are
// unrolled, so no lattice table lives in device memory.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tlbm_dev {

// ------------------------------------------------------------------ lattices

template <int Q>
struct Lat;

// D2Q9: rest, axis directions 1-4, diagonals 5-8 (opposites adjacent).
template <>
struct Lat<9> {
    static constexpr int D = 2;
    static constexpr int NAXIS = 4;
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int v[9] = {0, 1, -1, 0, 0, 1, -1, -1, 1};
        return v[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int v[9] = {0, 0, 0, 1, -1, 1, -1, 1, -1};
        return v[i];
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

// D3Q19 in the order the paper's weight table implies: rest; +-x, +-y, +-z;
// xy-plane edges 7-10; yz-plane edges 11-14; zx-plane edges 15-18.
template <>
struct Lat<19> {
    static constexpr int D = 3;
    static constexpr int NAXIS = 6;
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int v[19] = {0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, 1, -1, -1};
        return v[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int v[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 0, 0, 0, 0};
        return v[i];
    }
    __host__ __device__ static constexpr int cz(int i) {
        constexpr int v[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
        return v[i];
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};

template <int Q>
__host__ __device__ constexpr int comp(int i, int a) {
    return a == 0 ? Lat<Q>::cx(i) : (a == 1 ? Lat<Q>::cy(i) : Lat<Q>::cz(i));
}

template <int Q>
__host__ __device__ constexpr int opp(int i) {
    for (int j = 0; j < Q; ++j)
        if (Lat<Q>::cx(j) == -Lat<Q>::cx(i) && Lat<Q>::cy(j) == -Lat<Q>::cy(i) &&
            Lat<Q>::cz(j) == -Lat<Q>::cz(i))
            return j;
    return -1;
}

template <int Q>
__host__ __device__ constexpr int speed2(int i) {
    return Lat<Q>::cx(i) * Lat<Q>::cx(i) + Lat<Q>::cy(i) * Lat<Q>::cy(i) +
           Lat<Q>::cz(i) * Lat<Q>::cz(i);
}

// Gradient-term tensor w_i^{ab}, component c in (xx, yy, zz, xy, yz, zx).
// The pressure tensor needs (1/c_s^2) sum_i w_i^{aa} e_ia^2 = 1/2,
// (1/c_s^2) sum_i w_i^{aa} e_ib^2 = -1/2 and (1/c_s^2) sum_i w_i^{ab} e_ia e_ib = 1.
// D3Q19 (paper's table): an axis link along a has w^{aa} = 5/36 and -1/9 on the
// other diagonal components; an edge in plane (a,b) has w^{aa} = w^{bb} = -1/72,
// 1/36 on the normal component and w^{ab} = e_a e_b / 12.
// D2Q9 (same normalisation): axis link w^{aa} = 1/9, w^{bb} = -1/18; diagonal
// link w^{xx} = w^{yy} = -1/72, w^{xy} = e_x e_y / 12.
template <int Q>
__host__ __device__ constexpr double tens(int i, int c) {
    if (i == 0) return 0.0;
    if (c < 3) {
        const int ea = comp<Q>(i, c);
        if (Lat<Q>::D == 2 && c == 2) return 0.0;
        if (speed2<Q>(i) == 1) {
            if (Lat<Q>::D == 2) return ea != 0 ? 1.0 / 9.0 : -1.0 / 18.0;
            return ea != 0 ? 5.0 / 36.0 : -1.0 / 9.0;
        }
        // diagonal / edge link
        if (Lat<Q>::D == 2) return -1.0 / 72.0;
        return ea != 0 ? -1.0 / 72.0 : 1.0 / 36.0;
    }
    const int a = c - 3, b = (c - 3 + 1) % 3;  // xy, yz, zx
    if (speed2<Q>(i) != 2) return 0.0;
    return comp<Q>(i, a) * comp<Q>(i, b) / 12.0;
}

// ------------------------------------------------------------------ storage

// Scalar conversions of the storage types (compute type T).
template <typename S>
struct Store;

template <>
struct Store<double> {
    using T = double;
    static __device__ __forceinline__ double get(double v) { return v; }
    static __device__ __forceinline__ double put(double v) { return v; }
};

template <>
struct Store<float> {
    using T = float;
    static __device__ __forceinline__ float get(float v) { return v; }
    static __device__ __forceinline__ float put(float v) { return v; }
};

template <>
struct Store<__half> {
    using T = float;
    static __device__ __forceinline__ float get(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half put(float v) { return __float2half_rn(v); }
    // a 32-bit lane word of two values (low half first)
    static __device__ __forceinline__ void get2(unsigned w, float& a, float& b) {
        const float2 v = __half22float2(*reinterpret_cast<const __half2*>(&w));
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ unsigned put2(float a, float b) {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const unsigned*>(&h);
    }
};

template <>
struct Store<__nv_bfloat16> {
    using T = float;
    static __device__ __forceinline__ float get(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 put(float v) { return __float2bfloat16_rn(v); }
    // a 32-bit lane word of two values (low half first)
    static __device__ __forceinline__ void get2(unsigned w, float& a, float& b) {
        const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ unsigned put2(float a, float b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const unsigned*>(&h);
    }
};

// ------------------------------------------------------------------ geometry

// Population layout: 32-node chunks along x.  All populations of the 32 nodes
// x = 32c .. 32c+31 of one row (row = y + ny*z) form one contiguous chunk of
// Fmt<Q,S>::CHUNK bytes at ((row * ncx + c) * CHUNK), ncx = ceil(nx / 32).
// Inside a chunk, each run holds one lane word per node, Fmt::ESZ bytes apart,
// so a node is one byte offset, chunk + lane * ESZ, and every population of it
// is that offset plus a constant.
//   FP64, and FP32 on D2Q9: 3Q runs of S, run s*Q + i for set s, direction i.
//   FP32 on D3Q19: 64-bit lane words of two values, paired as in the 16-bit
//     formats below ((f_i, g_i), (k_i, k_opp(i))), and the rest populations as
//     (f_0, g_0) and (k_0, unused).  FP32 keeps f as its deviation f_i - w_i
//     from the rest state at rho = 1 (g and k as they are): deviations are
//     small, so FP32 rounding of the stored values, and with it the drift of
//     the total momentum, is ~100x smaller.
//   16-bit formats (packed): f is kept as its deviation f_i - w_i from the
//     rest state at rho = 1, g and k as they are.  Every lane word is 32 bits:
//     for each moving direction i one run of (f_i, g_i) pairs (the two share a
//     pull source: one load), for each pair of opposite directions i < opp(i)
//     one run of (k_i, k_opp(i)) pairs (the collision writes both at once: one
//     store), and three FP32 runs of the rest populations f_0 - w_0, g_0, k_0.
//     That is 3(Q-1) 16-bit values and three FP32 values per node, as dense as
//     16 bits allow.  The rest populations carry nearly all of phi and psi,
//     which 16 bits would round by up to 2.4e-4 per step; the moving
//     populations are small.  A collision writes each rest population as the
//     node's moment minus the moving populations as stored (rounded), so the
//     16-bit rounding moves mass between directions of a node but never changes
//     it; rho - 1 is summed from the small deviations, which keeps FP32
//     rounding from biasing the totals.
// A warp on 32 consecutive x of one row therefore finds all populations of its
// nodes in one chunk: each load or store is one base address plus an immediate
// offset.  Padding nodes (x >= nx in the last chunk) are never read or written.
struct Geom {
    int nx, ny, nz;
    long long N;   // nodes
    long long Np;  // stride of node-indexed moment arrays (N rounded up to 64)
    int ncx;       // 32-node chunks per row
};

template <int Q, typename S>
struct Fmt {
    using T = typename Store<S>::T;
    static constexpr bool PACKED = sizeof(S) == 2;
    // f kept as its deviation f_i - w_i from the rest state at rho = 1 (FP32 and
    // the 16-bit formats; FP64 stores f as it is)
    static constexpr bool OFFSET = sizeof(S) <= 4;
    // lane words of two values: the 16-bit formats, and FP32 on D3Q19 (measured:
    // 0.5 % faster there; on D2Q9, whose kernels run near the HBM limit, the
    // unused fourth word of the FP32 rest populations costs 5 %); FP64 one value
    static constexpr bool PAIRED = sizeof(S) == 2 || (sizeof(S) == 4 && Q == 19);
    static constexpr int VSZ = (int)sizeof(S);              // bytes of one value
    static constexpr int ESZ = PAIRED ? 2 * VSZ : VSZ;       // bytes between lanes of a run
    static constexpr int RUN = 32 * ESZ;                     // bytes of a run
    static constexpr int NKP = (Q - 1) / 2;                  // runs of k pairs
    // runs of the rest populations: 16-bit formats one FP32 word each; FP32 the
    // words (f_0, g_0) and (k_0, unused)
    static constexpr int NREST = PACKED ? 3 : 2;
    static constexpr long long CHUNK = PAIRED ? (long long)((Q - 1) + NKP + NREST) * RUN : 3LL * Q * 32 * ESZ;
    // packed: run of the k pair of direction i (the pairs of opposite directions
    // numbered by their lower direction), and the half of its lane word (0: i is
    // the lower direction of its pair).  Tables, so that they fold to immediates.
    __host__ __device__ static constexpr int kpair(int i) {
        if (Q == 19) {
            // pairs (1,2) (3,4) (5,6) (7,10) (8,9) (11,14) (12,13) (15,18) (16,17)
            constexpr int v[19] = {0, 0, 0, 1, 1, 2, 2, 3, 4, 4, 3, 5, 6, 6, 5, 7, 8, 8, 7};
            return v[i];
        }
        // D2Q9: opposites adjacent, pairs (1,2) (3,4) (5,6) (7,8)
        return (i - 1) / 2;
    }
    __host__ __device__ static constexpr int khalf(int i) {
        if (Q == 19) {
            constexpr int v[19] = {0, 0, 1, 0, 1, 0, 1, 0, 0, 1, 1, 0, 0, 1, 1, 0, 0, 1, 1};
            return v[i];
        }
        return (i - 1) & 1;
    }
    // byte offset of (s, i) in the lane word of lane 0
    __host__ __device__ static constexpr int off(int s, int i) {
        if (!PAIRED) return (s * Q + i) * 32 * ESZ;
        if (i == 0) {
            if (PACKED) return ((Q - 1) + NKP + s) * RUN;
            return ((Q - 1) + NKP + (s == 2 ? 1 : 0)) * RUN + (s == 1 ? 4 : 0);
        }
        if (s < 2) return (i - 1) * RUN + s * VSZ;
        return ((Q - 1) + kpair(i)) * RUN + khalf(i) * VSZ;
    }
    // rest-state value subtracted before storage (set f, offset formats)
    __host__ __device__ static constexpr double bias(int s, int i) {
        return (OFFSET && s == 0) ? Lat<Q>::w(i) : 0.0;
    }
    // stored value of (s, i) at node pointer n (chunk + lane * ESZ): x - bias
    static __device__ __forceinline__ T ld_delta(const unsigned char* n, int s, int i) {
        if constexpr (PACKED) {
            if (i == 0) return *reinterpret_cast<const float*>(n + off(s, 0));
            return Store<S>::get(*reinterpret_cast<const S*>(n + off(s, i)));
        } else {
            return *reinterpret_cast<const S*>(n + off(s, i));
        }
    }
    // value from its stored deviation and back (no add where the bias is zero:
    // x + 0 is not x for x = -0, so the compiler would keep it)
    static __device__ __forceinline__ T unbias(int s, int i, T d) {
        const double b = bias(s, i);
        return b == 0.0 ? d : d + T(b);
    }
    static __device__ __forceinline__ T dev(int s, int i, T v) {
        const double b = bias(s, i);
        return b == 0.0 ? v : v - T(b);
    }
    // population (s, i) at node pointer n
    static __device__ __forceinline__ T ld(const unsigned char* n, int s, int i) {
        const double b = bias(s, i);
        return b == 0.0 ? ld_delta(n, s, i) : ld_delta(n, s, i) + T(b);
    }
    // the same, marking the line evict-first (its last use in this kernel)
    static __device__ __forceinline__ T ld_last(const unsigned char* n, int s, int i) {
        const double b = bias(s, i);
        return b == 0.0 ? ld_last_delta(n, s, i) : ld_last_delta(n, s, i) + T(b);
    }
    // stored value of (s, i), marking the line evict-first (its last use)
    static __device__ __forceinline__ T ld_last_delta(const unsigned char* n, int s, int i) {
        if constexpr (PACKED) {
            if (i == 0) return __ldcs(reinterpret_cast<const float*>(n + off(s, 0)));
            return Store<S>::get(__ldcs(reinterpret_cast<const S*>(n + off(s, i))));
        } else {
            return __ldcs(reinterpret_cast<const S*>(n + off(s, i)));
        }
    }
    // stored values of f_i and g_i, i >= 1, at node pointer n (packed: one load
    // of their lane word; LAST marks it evict-first)
    template <bool LAST = false>
    static __device__ __forceinline__ void ld_fg(const unsigned char* n, int i, T& f, T& g) {
        if constexpr (PACKED) {
            const unsigned* p = reinterpret_cast<const unsigned*>(n + off(0, i));
            Store<S>::get2(LAST ? __ldcs(p) : *p, f, g);
        } else if constexpr (PAIRED) {
            const float2* p = reinterpret_cast<const float2*>(n + off(0, i));
            const float2 v = LAST ? __ldcs(p) : *p;
            f = v.x;
            g = v.y;
        } else {
            f = LAST ? ld_last_delta(n, 0, i) : ld_delta(n, 0, i);
            g = LAST ? ld_last_delta(n, 1, i) : ld_delta(n, 1, i);
        }
    }
    // store the deviation d of (s, i) with an evict-first hint
    static __device__ __forceinline__ void st_stream_delta(unsigned char* n, int s, int i, T d) {
        if constexpr (PACKED) {
            if (i == 0) __stcs(reinterpret_cast<float*>(n + off(s, 0)), d);
            else __stcs(reinterpret_cast<S*>(n + off(s, i)), Store<S>::put(d));
        } else {
            __stcs(reinterpret_cast<S*>(n + off(s, i)), d);
        }
    }
    // the deviation a store of deviation d leaves in memory, as read back
    static __device__ __forceinline__ T qdelta_d(int i, T d) {
        if constexpr (PACKED) {
            if (i > 0) return Store<S>::get(Store<S>::put(d));
        }
        return d;
    }
    // store with an evict-first hint (streamed out, read only by the next step)
    static __device__ __forceinline__ void st_stream(unsigned char* n, int s, int i, T v) {
        const double b = bias(s, i);
        st_stream_delta(n, s, i, b == 0.0 ? v : v - T(b));
    }
    // store the deviation d = x - bias of (s, i)
    static __device__ __forceinline__ void st_delta(unsigned char* n, int s, int i, T d) {
        if constexpr (PACKED) {
            if (i == 0) *reinterpret_cast<float*>(n + off(s, 0)) = d;
            else *reinterpret_cast<S*>(n + off(s, i)) = Store<S>::put(d);
        } else {
            *reinterpret_cast<S*>(n + off(s, i)) = d;
        }
    }
    static __device__ __forceinline__ void st(unsigned char* n, int s, int i, T v) {
        const double b = bias(s, i);
        st_delta(n, s, i, b == 0.0 ? v : v - T(b));
    }
    // store the deviations of f_i, g_i (i >= 1) and, in a second call, of k_i and
    // k_o for o = opp(i) (packed: one 32-bit store each; STREAM: evict-first)
    template <bool STREAM>
    static __device__ __forceinline__ void st_fg(unsigned char* n, int i, T df, T dg) {
        if constexpr (PACKED) {
            unsigned* p = reinterpret_cast<unsigned*>(n + off(0, i));
            const unsigned w = Store<S>::put2(df, dg);
            if (STREAM) __stcs(p, w);
            else *p = w;
        } else if constexpr (PAIRED) {
            float2* p = reinterpret_cast<float2*>(n + off(0, i));
            const float2 w = make_float2(df, dg);
            if (STREAM) __stcs(p, w);
            else *p = w;
        } else if (STREAM) {
            st_stream_delta(n, 0, i, df);
            st_stream_delta(n, 1, i, dg);
        } else {
            st_delta(n, 0, i, df);
            st_delta(n, 1, i, dg);
        }
    }
    template <bool STREAM>
    static __device__ __forceinline__ void st_kk(unsigned char* n, int i, T dki, T dko) {
        if constexpr (PACKED) {
            const bool lo = khalf(i) == 0;  // the lower direction sits in the low half
            unsigned* p = reinterpret_cast<unsigned*>(n + off(2, lo ? i : opp<Q>(i)));
            const unsigned w = lo ? Store<S>::put2(dki, dko) : Store<S>::put2(dko, dki);
            if (STREAM) __stcs(p, w);
            else *p = w;
        } else if constexpr (PAIRED) {
            const bool lo = khalf(i) == 0;
            float2* p = reinterpret_cast<float2*>(n + off(2, lo ? i : opp<Q>(i)));
            const float2 w = lo ? make_float2(dki, dko) : make_float2(dko, dki);
            if (STREAM) __stcs(p, w);
            else *p = w;
        } else if (STREAM) {
            st_stream_delta(n, 2, i, dki);
            st_stream_delta(n, 2, opp<Q>(i), dko);
        } else {
            st_delta(n, 2, i, dki);
            st_delta(n, 2, opp<Q>(i), dko);
        }
    }
    // st_fg / st_kk that also return the deviations as stored (read back from
    // the lane word itself: no second conversion of each value)
    template <bool STREAM>
    static __device__ __forceinline__ void st_fg_q(unsigned char* n, int i, T df, T dg, T& qf, T& qg) {
        if constexpr (PACKED) {
            unsigned* p = reinterpret_cast<unsigned*>(n + off(0, i));
            const unsigned w = Store<S>::put2(df, dg);
            if (STREAM) __stcs(p, w);
            else *p = w;
            Store<S>::get2(w, qf, qg);
        } else {
            st_fg<STREAM>(n, i, df, dg);
            qf = df;
            qg = dg;
        }
    }
    template <bool STREAM>
    static __device__ __forceinline__ void st_kk_q(unsigned char* n, int i, T dki, T dko, T& qi, T& qo) {
        if constexpr (PACKED) {
            const bool lo = khalf(i) == 0;
            unsigned* p = reinterpret_cast<unsigned*>(n + off(2, lo ? i : opp<Q>(i)));
            const unsigned w = lo ? Store<S>::put2(dki, dko) : Store<S>::put2(dko, dki);
            if (STREAM) __stcs(p, w);
            else *p = w;
            if (lo) Store<S>::get2(w, qi, qo);
            else Store<S>::get2(w, qo, qi);
        } else {
            st_kk<STREAM>(n, i, dki, dko);
            qi = dki;
            qo = dko;
        }
    }
    // the deviation a store of population value v leaves in memory, as read back
    static __device__ __forceinline__ T qdelta(int s, int i, T v) {
        const double b = bias(s, i);
        const T d = b == 0.0 ? v : v - T(b);
        if constexpr (PACKED) {
            if (i > 0) return Store<S>::get(Store<S>::put(d));
        }
        return d;
    }
};

// byte offset of node (x, y, z) in a population buffer: its chunk plus its lane
template <int Q, typename S>
__host__ __device__ __forceinline__ long long node_off(const Geom& g, int x, int y, int z) {
    const long long row = (long long)y + (long long)g.ny * z;
    return (row * g.ncx + (x >> 5)) * Fmt<Q, S>::CHUNK + (x & 31) * Fmt<Q, S>::ESZ;
}

template <int Q, typename S>
__device__ __forceinline__ typename Store<S>::T pld(const void* base, const Geom& g, int s, int i, int x,
                                                    int y, int z) {
    return Fmt<Q, S>::ld(static_cast<const unsigned char*>(base) + node_off<Q, S>(g, x, y, z), s, i);
}

template <int Q, typename S>
__device__ __forceinline__ void pst(void* base, const Geom& g, int s, int i, int x, int y, int z,
                                    typename Store<S>::T v) {
    Fmt<Q, S>::st(static_cast<unsigned char*>(base) + node_off<Q, S>(g, x, y, z), s, i, v);
}

// raw store (no rest-state offset): arrays in the population layout that hold
// something other than populations (the adjoint's multipliers)
template <int Q, typename S>
__device__ __forceinline__ void pst_raw(void* base, const Geom& g, int s, int i, int x, int y, int z,
                                        typename Store<S>::T v) {
    Fmt<Q, S>::st_delta(static_cast<unsigned char*>(base) + node_off<Q, S>(g, x, y, z), s, i, v);
}

__device__ __forceinline__ int wrap(int v, int n) {
    v += (v < 0) ? n : 0;
    v -= (v >= n) ? n : 0;
    return v;
}

__device__ __forceinline__ long long node(const Geom& g, int x, int y, int z) {
    return (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * (long long)z);
}

// --------------------------------------------------------------- parameters

template <typename T>
struct Phys {
    T kappa[3];  // kappa_1..3
    T a2;        // alpha^2
    T omega[3];  // 1/tau for f, g, k
    T gamma[2];  // Gamma_phi, Gamma_psi
    T Gw[3];     // wall-normal gradients of rho, phi, psi (wetting condition)
    T K[3][3];   // mixing coefficients kappa_XY of the pressure tensor
};

// ------------------------------------------------------------- node physics

// Per-node quantities from which every equilibrium population follows:
//   f_eq_i = w_i (bf + 3 e_i.j + 9/2 rho (e_i.u)^2) + sum_c w_i^c Gs_c
//   g_eq_i = w_i (bg + 3 phi e_i.u + 9/2 phi (e_i.u)^2)       (k_eq likewise)
// with bf = 3 p_b - 3 alpha^2 L - 3/2 rho u^2, bg = 3 Gamma_phi mu_phi - 3/2 phi u^2,
// bk = 3 Gamma_psi mu_psi - 3/2 psi u^2 and Gs_c = 3 alpha^2 G_c (c_s^2 = 1/3).
template <int Q, typename T>
struct NodeEq {
    T rho, phi, psi;
    T ux, uy, uz;
    T bf, bg, bk;
    T bf1;  // bf - 1, from rho - 1 without cancellation (when setup gets rd)
    T Gs[6];

    // X = (rho, phi, psi), j = rho u, grad[X][a], lap[X]; rd = rho - 1 as summed
    // from stored f deviations (the offset formats), used for bf1
    __host__ __device__ __forceinline__ void setup(const Phys<T>& P, T rho_, T jx, T jy, T jz, T phi_,
                                          T psi_, const T (&grad)[3][3], const T (&lap)[3], T rd = T(0)) {
        rho = rho_; phi = phi_; psi = psi_;
        const T inv = T(1) / rho;
        ux = jx * inv; uy = jy * inv; uz = jz * inv;
        const T uu = ux * ux + uy * uy + uz * uz;
        // concentrations and their Laplacians (Sec. Auxiliary variables)
        const T C[3] = {(rho + phi - psi) * T(0.5), (rho - phi - psi) * T(0.5), psi};
        const T lC[3] = {(lap[0] + lap[1] - lap[2]) * T(0.5), (lap[0] - lap[1] - lap[2]) * T(0.5),
                         lap[2]};
        T mu[3];
        T pbx = T(0);  // p_b - rho c_s^2
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const T c = C[m];
            const T c1 = T(1) - c;
            mu[m] = P.kappa[m] * (c * c1 * (T(1) - T(2) * c) - P.a2 * lC[m]);
            pbx += P.kappa[m] * T(0.5) * c * c * c1 * (T(1) - T(3) * c);
        }
        const T pb = rho * T(1.0 / 3.0) + pbx;
        const T mu_phi = (mu[0] - mu[1]) * T(0.5);
        const T mu_psi = mu[2] - (mu[0] + mu[1]) * T(0.5);
        // Laplacian part of the pressure tensor: L = sum_XY K_XY X lap Y
        const T X[3] = {rho, phi, psi};
        T Lp = T(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            T s = T(0);
#pragma unroll
            for (int b = 0; b < 3; ++b) s += P.K[a][b] * lap[b];
            Lp += X[a] * s;
        }
        bf = T(3) * pb - T(3) * P.a2 * Lp - T(1.5) * rho * uu;
        bf1 = (T(3) * pbx + rd) - T(3) * P.a2 * Lp - T(1.5) * rho * uu;
        bg = T(3) * P.gamma[0] * mu_phi - T(1.5) * phi * uu;
        bk = T(3) * P.gamma[1] * mu_psi - T(1.5) * psi * uu;
        // gradient part: G_ab = v_a^T K v_b with v_a = (d_a rho, d_a phi, d_a psi)
        constexpr int D = Lat<Q>::D;
        T Kv[3][3];  // [b][X] = (K v_b)_X
#pragma unroll
        for (int b = 0; b < D; ++b)
#pragma unroll
            for (int x = 0; x < 3; ++x)
                Kv[b][x] = P.K[x][0] * grad[0][b] + P.K[x][1] * grad[1][b] + P.K[x][2] * grad[2][b];
        const T s3 = T(3) * P.a2;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const int a = c < 3 ? c : c - 3;
            const int b = c < 3 ? c : (c - 3 + 1) % 3;
            if (a < D && b < D)
                Gs[c] = s3 * (grad[0][a] * Kv[b][0] + grad[1][a] * Kv[b][1] + grad[2][a] * Kv[b][2]);
            else
                Gs[c] = T(0);
        }
    }

    __host__ __device__ __forceinline__ T eu(int i) const {
        T s = T(0);
        if (Lat<Q>::cx(i)) s += T(Lat<Q>::cx(i)) * ux;
        if (Lat<Q>::cy(i)) s += T(Lat<Q>::cy(i)) * uy;
        if (Lat<Q>::cz(i)) s += T(Lat<Q>::cz(i)) * uz;
        return s;
    }

    __host__ __device__ __forceinline__ T grad_term(int i) const {
        T s = T(0);
#pragma unroll
        for (int c = 0; c < 6; ++c)
            if (tens<Q>(i, c) != 0.0) s += T(tens<Q>(i, c)) * Gs[c];
        return s;
    }

    // equilibria of direction i >= 1
    __host__ __device__ __forceinline__ void eq(int i, T& fe, T& ge, T& ke) const {
        const T w = T(Lat<Q>::w(i));
        const T e = eu(i);
        const T e2 = T(4.5) * e * e;
        fe = w * (bf + rho * (T(3) * e + e2)) + grad_term(i);
        ge = w * (bg + phi * (T(3) * e + e2));
        ke = w * (bk + psi * (T(3) * e + e2));
    }
};

}  // namespace tlbm_dev
