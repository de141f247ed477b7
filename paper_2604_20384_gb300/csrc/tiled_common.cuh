// Device helpers of the window-pass kernels, shared by the per-pass kernels
// (tiled.cu), the two-direction kernels (pair.cu) and the persistent batch
// kernel (batch.cu): tile I/O, bulk copies with mbarriers, gate arithmetic,
// warp reductions. See tiled.cu for the arithmetic of a pass.
#pragma once

#include "internal.h"

namespace hvp {
namespace tile {

__device__ __forceinline__ unsigned insert0(unsigned x, int p) {
    return ((x >> p) << (p + 1)) | (x & ((1u << p) - 1u));
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float2 swp(float2 x) { return make_float2(x.y, x.x); }

// ---------------------------------------------------------------- arithmetic
// Matrix element storage: scalar form keeps float2 {re, im}; packed form keeps
// float4 {re, re, -im, im} so that acc += m x is
//     acc = fma2({re, re}, {x.re, x.im}, acc); acc = fma2({-im, im}, {x.im, x.re}, acc).
template <bool P2>
struct Math;

template <>
struct Math<false> {
    using M = float2;
    static constexpr int kMatBytes = 8;
    __device__ static __forceinline__ void mac(float2& acc, const M& m, float2 x, float2 /*xs*/) {
        acc.x = fmaf(m.x, x.x, acc.x);
        acc.x = fmaf(-m.y, x.y, acc.x);
        acc.y = fmaf(m.x, x.y, acc.y);
        acc.y = fmaf(m.y, x.x, acc.y);
    }
    __device__ static __forceinline__ void msub(float2& acc, const M& m, float2 x, float2 /*xs*/) {  // acc -= m x
        acc.x = fmaf(-m.x, x.x, acc.x);
        acc.x = fmaf(m.y, x.y, acc.x);
        acc.y = fmaf(-m.x, x.y, acc.y);
        acc.y = fmaf(-m.y, x.x, acc.y);
    }
    // acc += conj(a) x; (ar, ai) = a as given, x and its swap
    __device__ static __forceinline__ void cmac(float2& acc, float2 a, float2 x, float2 /*xs*/) {
        acc.x = fmaf(a.x, x.x, acc.x);
        acc.x = fmaf(a.y, x.y, acc.x);
        acc.y = fmaf(a.x, x.y, acc.y);
        acc.y = fmaf(-a.y, x.x, acc.y);
    }
    __device__ static __forceinline__ M expand(float2 m) { return m; }
};

template <>
struct Math<true> {
    using M = float4;
    static constexpr int kMatBytes = 16;
    __device__ static __forceinline__ void mac(float2& acc, const M& m, float2 x, float2 xs) {
        acc = __ffma2_rn(make_float2(m.x, m.y), x, acc);
        acc = __ffma2_rn(make_float2(m.z, m.w), xs, acc);
    }
    __device__ static __forceinline__ void msub(float2& acc, const M& m, float2 x, float2 xs) {
        acc = __ffma2_rn(make_float2(-m.x, -m.y), x, acc);
        acc = __ffma2_rn(make_float2(-m.z, -m.w), xs, acc);
    }
    // acc += conj(a) x = {a.re, a.re} x + {a.im, -a.im} swap(x)
    __device__ static __forceinline__ void cmac(float2& acc, float2 a, float2 x, float2 xs) {
        acc = __ffma2_rn(make_float2(a.x, a.x), x, acc);
        acc = __ffma2_rn(make_float2(a.y, -a.y), xs, acc);
    }
    __device__ static __forceinline__ M expand(float2 m) { return make_float4(m.x, m.x, -m.y, m.y); }
};

// y = M x for a 4x4 complex matrix in shared memory (row-major).
template <bool P2, class MA>
__device__ __forceinline__ void matvec4(MA M, const float2 (&x)[4], const float2 (&xs)[4], float2 (&y)[4]) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 4; ++c) Math<P2>::mac(acc, M[r * 4 + c], x[c], xs[c]);
        y[r] = acc;
    }
}

template <bool P2>
__device__ __forceinline__ void swaps(const float2 (&x)[4], float2 (&xs)[4]) {
#pragma unroll
    for (int c = 0; c < 4; ++c) xs[c] = P2 ? swp(x[c]) : x[c];
}

// Reduce-scatter of NV values over a warp: afterwards lane l holds in v[0..NV/32)
// the warp sums of components l*(NV/32) + i.
template <int NV>
__device__ __forceinline__ void warp_reduce_scatter(float (&v)[NV], int lane) {
#pragma unroll
    for (int step = 0; step < 5; ++step) {
        const int off = 16 >> step;
        const int half = (NV >> step) / 2;
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            float send = up ? v[i] : v[i + half];
            float keep = up ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
}

template <bool TAN>
struct Elt;
template <>
struct Elt<true> { using T = float4; };
template <>
struct Elt<false> { using T = float2; };

__device__ __forceinline__ float2 lo2(float4 x) { return make_float2(x.x, x.y); }
__device__ __forceinline__ float2 hi2(float4 x) { return make_float2(x.z, x.w); }

// Matrix slots per gate in shared memory: forward kernel {G, V}; backward
// kernel {G^-1, G^dag, V, V^dag} and, in the turnaround pass, also G.
constexpr int kFwdMats = 2;

// ------------------------------------------------------------ tile I/O
struct TileCtx {
    size_t base;
    const uint32_t* offlo;
    const uint32_t* offhi;
};

// ------------------------------------------------- bulk copies and mbarriers
// One-dimensional bulk copies (cp.async.bulk, the TMA engine without a tensor
// map) from global into shared memory, completed on an mbarrier by byte
// count. Sizes and both addresses are multiples of 16 bytes.
__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes initialised mbarriers and earlier generic-proxy shared-memory accesses
// of this thread visible to the async proxy (bulk copies).
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The barrier is told to expect `bytes + extra` bytes: extra = 0 in normal
// use; a positive extra keeps the phase from completing (test of the bounded
// waits).
__device__ __forceinline__ void bulk_load_async(void* dst, const void* src, unsigned bytes, uint64_t* bar,
                                                unsigned extra = 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes + extra)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits until the barrier's phase with the given parity has completed; gives
// up (returns false) after `limit` polls, the later ones 256 ns apart
// (limit = 1 << 23: about two seconds).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned limit) {
    for (unsigned i = 0; i < limit; ++i) {
        if (mbar_test(bar, parity)) return true;
        if (i >= 64) __nanosleep(256);
    }
    return false;
}

// Tile t of sample s in slot `slot` of the forward cache (slot k: the forward
// states before gate k in pass order), one contiguous block of 2^w elements
// in shared-memory order.
template <typename E>
__device__ __forceinline__ E* cache_tile(const TiledArgs& a, int slot, int s, unsigned t, int ng, int Lt) {
    return reinterpret_cast<E*>(static_cast<char*>(a.cache) + (size_t)slot * a.cache_slot_bytes) +
           (((size_t)s << ng) + t) * (size_t)Lt;
}

__device__ __forceinline__ size_t tile_base(const DevPass* __restrict__ P, unsigned t, size_t sample_off, int ng) {
    size_t base = sample_off;
    for (int r = 0; r < ng; ++r)
        if ((t >> r) & 1u) base |= (size_t)1 << __ldg(&P->gpos[r]);
    return base;
}

// CG: read through L2 only (data written by other CTAs of the same launch).
template <typename E>
__device__ __forceinline__ E ld_state(const E* p, bool cg) {
    if (cg) return __ldcg(p);
    return *p;
}

template <typename E, int NT, bool CG = false>
__device__ __forceinline__ void load_tile(E* __restrict__ dst, const E* __restrict__ src, const TileCtx& tc,
                                          const uint16_t* lo, const uint16_t* hi, int Lt) {
    for (int m = threadIdx.x; m < Lt; m += NT) {
        const size_t addr = tc.base + __ldg(&tc.offlo[m & 63]) + __ldg(&tc.offhi[m >> 6]);
        const unsigned l = __ldg(&lo[m & 63]) | __ldg(&hi[m >> 6]);
        dst[swz(l)] = ld_state(src + addr, CG);
    }
}

template <typename E, int NT>
__device__ __forceinline__ void store_tile(E* __restrict__ dst, const E* __restrict__ src, const TileCtx& tc,
                                           const uint16_t* lo, const uint16_t* hi, int Lt) {
    for (int m = threadIdx.x; m < Lt; m += NT) {
        const size_t addr = tc.base + __ldg(&tc.offlo[m & 63]) + __ldg(&tc.offhi[m >> 6]);
        const unsigned l = __ldg(&lo[m & 63]) | __ldg(&hi[m >> 6]);
        dst[addr] = src[swz(l)];
    }
}

// psi^[0] = (x)_q psi_{s,q}: tile factor of the fixed qubits times the factors
// of the window qubits (Eq. costHS, product states). q1 points at the tile's
// first sample; local index bits at and above nq select further samples
// (several small samples packed into one tile), each n qubits apart.
template <typename E, int NT>
__device__ __forceinline__ void gen_tile(E* __restrict__ sf, const DevPass* __restrict__ P, const float2* q1,
                                         unsigned t, int nq, int ng, int Lt, int n) {
    float2 gamma = make_float2(1.f, 0.f);
    for (int r = 0; r < ng; ++r) gamma = cmulf(gamma, __ldg(&q1[2 * __ldg(&P->gq[r]) + ((t >> r) & 1u)]));
    for (int l = threadIdx.x; l < Lt; l += NT) {
        const float2* qs = q1 + (size_t)(l >> nq) * 2 * n;
        float2 amp = gamma;
        for (int j = 0; j < nq; ++j) amp = cmulf(amp, __ldg(&qs[2 * __ldg(&P->sq[j]) + ((l >> j) & 1)]));
        if constexpr (sizeof(E) == 16) sf[swz(l)] = E{amp.x, amp.y, 0.f, 0.f};
        else sf[swz(l)] = amp;
    }
}

// Stage matrices of the pass's gates into shared memory (expanded for the
// packed form): nmat slots per gate, slot i holding Mats32 field which[i]
// (fields: 0 G, 1 G^-1, 2 G^dag, 3 V, 4 V^dag).
template <bool P2, int NT>
__device__ __forceinline__ void stage_mats(typename Math<P2>::M* __restrict__ dst, const TiledArgs& a, int goff,
                                           int ngates, int nmat, const int* which) {
    for (int i = threadIdx.x; i < ngates * nmat * 16; i += NT) {
        const int g = i / (nmat * 16), rem = i - g * nmat * 16, mi = rem >> 4, e = rem & 15;
        const int k = __ldg(&a.gates[goff + g].k);
        const float2 v = reinterpret_cast<const float2*>(a.mats + k)[which[mi] * 16 + e];
        dst[i] = Math<P2>::expand(v);
    }
}

// One forward gate over all groups of the tile.
// MA: matrix accessor (a pointer into shared memory, or any type with
// operator[] returning a matrix element).
// Number of groups a thread handles in one gate: GPT when it is fixed at
// compile time (the loop then unrolls), else from the tile size.
template <int NT, int GPT>
__device__ __forceinline__ int groups_of_thread(int Lt) {
    if constexpr (GPT > 0) return GPT;
    return ((Lt >> 2) + NT - 1 - (int)threadIdx.x) / NT;
}

// Shared-memory slots of the four amplitudes of a thread's it-th group of a
// gate on index bits u, v (plo < phi_): group q = tid + it * NT spreads over
// the index bits other than plo and phi_. With GPT fixed, q's bits above
// log2(NT) come from `it` alone and land on index bits >= 8 (NT = 256), which
// the swizzle does not touch, so the slots are those of group tid OR-ed with
// a per-iteration constant.
template <int NT, int GPT>
struct GroupIndex {
    unsigned base[4];
    unsigned d[GPT > 0 ? GPT : 1];
    int tid, plo, phi_;
    unsigned mu, mv;
    __device__ __forceinline__ GroupIndex(int t, int lo, int hi, unsigned u, unsigned v)
        : tid(t), plo(lo), phi_(hi), mu(u), mv(v) {
        if constexpr (GPT > 0) {
            const unsigned l0 = insert0(insert0(t, lo), hi);
            base[0] = swz(l0); base[1] = swz(l0 | v); base[2] = swz(l0 | u); base[3] = swz(l0 | u | v);
#pragma unroll
            for (int k = 0; k < GPT; ++k) d[k] = insert0(insert0(k * NT, lo), hi);
        }
    }
    __device__ __forceinline__ void get(int it, unsigned (&idx)[4]) const {
        if constexpr (GPT > 0) {
#pragma unroll
            for (int c = 0; c < 4; ++c) idx[c] = base[c] | d[it];
        } else {
            const unsigned l0 = insert0(insert0(tid + it * NT, plo), phi_);
            idx[0] = swz(l0); idx[1] = swz(l0 | mv); idx[2] = swz(l0 | mu); idx[3] = swz(l0 | mu | mv);
        }
    }
};

// With DUMP, the states after the gate are also written to `dump` (global
// memory, same element order as the shared-memory tile).
template <bool TAN, bool P2, int NT, class MA = const typename Math<P2>::M*, int GPT = 0, bool DUMP = false>
__device__ __forceinline__ void fwd_gate(typename Elt<TAN>::T* __restrict__ sf, MA Gm_s, MA Vm_s, int u, int v,
                                         int Lt, typename Elt<TAN>::T* __restrict__ dump = nullptr) {
    const int plo = min(u, v), phi_ = max(u, v);
    const unsigned mu = 1u << u, mv = 1u << v;
    // The gate's matrices are read from shared memory once per thread and
    // kept in registers for all of the thread's groups.
    using MT = typename Math<P2>::M;
    MT Gm[16], Vm[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        Gm[e] = Gm_s[e];
        if constexpr (TAN) Vm[e] = Vm_s[e];
    }
    const int ng = groups_of_thread<NT, GPT>(Lt);
    GroupIndex<NT, GPT> gi(threadIdx.x, plo, phi_, mu, mv);
#pragma unroll
    for (int it = 0; it < ng; ++it) {
        unsigned idx[4];
        gi.get(it, idx);
        if constexpr (TAN) {
            float2 p[4], d[4], ps[4], ds[4], np[4], nd[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) { const float4 x = sf[idx[c]]; p[c] = lo2(x); d[c] = hi2(x); }
            swaps<P2>(p, ps);
            swaps<P2>(d, ds);
            matvec4<P2>(Gm, p, ps, np);
            matvec4<P2>(Gm, d, ds, nd);
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) Math<P2>::mac(nd[r], Vm[r * 4 + c], p[c], ps[c]);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float4 o = make_float4(np[r].x, np[r].y, nd[r].x, nd[r].y);
                sf[idx[r]] = o;
                if constexpr (DUMP) dump[idx[r]] = o;
            }
        } else {
            float2 p[4], ps[4], np[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) p[c] = sf[idx[c]];
            swaps<P2>(p, ps);
            matvec4<P2>(Gm, p, ps, np);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                sf[idx[r]] = np[r];
                if constexpr (DUMP) dump[idx[r]] = np[r];
            }
        }
    }
}


// One backward gate over all groups of the tile: recompute the forward states
// before the gate (Vm holds Y = G^-1 V G^-1), add the gate's environment sums
// to red[] (E then DE, real and imaginary parts interleaved), update the
// co-states.
template <bool TAN, bool P2, int NT, int NV, class MA = const typename Math<P2>::M*, int GPT = 0>
__device__ __forceinline__ void bwd_gate(typename Elt<TAN>::T* __restrict__ sf, typename Elt<TAN>::T* __restrict__ sb,
                                         MA Gi, MA Gh, MA Vm, MA Vh, int u, int v, int Lt, float (&red)[NV]) {
    const int tid = threadIdx.x;
    const int plo = min(u, v), phi_ = max(u, v);
    const unsigned mu = 1u << u, mv = 1u << v;
    const int ng = groups_of_thread<NT, GPT>(Lt);
    GroupIndex<NT, GPT> gi(tid, plo, phi_, mu, mv);
#pragma unroll
    for (int it = 0; it < ng; ++it) {
        unsigned idx[4];
        gi.get(it, idx);
        if constexpr (TAN) {
            float2 p[4], d[4], A[4], B[4], xs[4], pp[4], pps[4], tt[4], dp[4], dps[4], nA[4], nB[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float4 x = sf[idx[c]];
                const float4 y = sb[idx[c]];
                p[c] = lo2(x); d[c] = hi2(x); A[c] = lo2(y); B[c] = hi2(y);
            }
            swaps<P2>(p, xs);
            swaps<P2>(d, tt);
            matvec4<P2>(Gi, p, xs, pp);                       // psi^[k-1] = G^-1 psi^[k]
            matvec4<P2>(Gi, d, tt, dp);                       // dpsi^[k-1] = G^-1 dpsi^[k] - Y psi^[k]
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) Math<P2>::msub(dp[r], Vm[r * 4 + c], p[c], xs[c]);
            swaps<P2>(pp, pps);
            swaps<P2>(dp, dps);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float2 e1 = make_float2(red[2 * (i * 4 + j)], red[2 * (i * 4 + j) + 1]);
                    Math<P2>::cmac(e1, A[i], pp[j], pps[j]);
                    red[2 * (i * 4 + j)] = e1.x;
                    red[2 * (i * 4 + j) + 1] = e1.y;
                    float2 e2 = make_float2(red[32 + 2 * (i * 4 + j)], red[32 + 2 * (i * 4 + j) + 1]);
                    Math<P2>::cmac(e2, B[i], pp[j], pps[j]);
                    Math<P2>::cmac(e2, A[i], dp[j], dps[j]);
                    red[32 + 2 * (i * 4 + j)] = e2.x;
                    red[32 + 2 * (i * 4 + j) + 1] = e2.y;
                }
            swaps<P2>(A, xs);
            matvec4<P2>(Gh, A, xs, nA);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                nB[r] = make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < 4; ++c) Math<P2>::mac(nB[r], Vh[r * 4 + c], A[c], xs[c]);
            }
            swaps<P2>(B, xs);
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) Math<P2>::mac(nB[r], Gh[r * 4 + c], B[c], xs[c]);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                sf[idx[r]] = make_float4(pp[r].x, pp[r].y, dp[r].x, dp[r].y);
                sb[idx[r]] = make_float4(nA[r].x, nA[r].y, nB[r].x, nB[r].y);
            }
        } else {
            float2 p[4], A[4], xs[4], pp[4], pps[4], nA[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) { p[c] = sf[idx[c]]; A[c] = sb[idx[c]]; }
            swaps<P2>(p, xs);
            matvec4<P2>(Gi, p, xs, pp);
            swaps<P2>(pp, pps);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float2 e1 = make_float2(red[2 * (i * 4 + j)], red[2 * (i * 4 + j) + 1]);
                    Math<P2>::cmac(e1, A[i], pp[j], pps[j]);
                    red[2 * (i * 4 + j)] = e1.x;
                    red[2 * (i * 4 + j) + 1] = e1.y;
                }
            swaps<P2>(A, xs);
            matvec4<P2>(Gh, A, xs, nA);
#pragma unroll
            for (int r = 0; r < 4; ++r) { sf[idx[r]] = pp[r]; sb[idx[r]] = nA[r]; }
        }
    }
}

// One backward gate with the forward states before the gate taken from a
// cache (sc: psi^[k-1], dpsi^[k-1] as written by the forward pass) instead of
// being recomputed: environment sums with the pre-update co-states, then the
// co-state update (Eq. environment, Eq. Dpsi, Eq. bis, Eq. dbis).
template <bool TAN, int NT, int NV, int GPT = 0>
__device__ __forceinline__ void bwd_gate_cached(const typename Elt<TAN>::T* __restrict__ sc,
                                                typename Elt<TAN>::T* __restrict__ sb, const float2* Gh,
                                                const float2* Vh, int u, int v, int Lt, float (&red)[NV]) {
    using M = Math<false>;
    const int plo = min(u, v), phi_ = max(u, v);
    const unsigned mu = 1u << u, mv = 1u << v;
    const int ng = groups_of_thread<NT, GPT>(Lt);
    GroupIndex<NT, GPT> gi(threadIdx.x, plo, phi_, mu, mv);
#pragma unroll
    for (int it = 0; it < ng; ++it) {
        unsigned idx[4];
        gi.get(it, idx);
        if constexpr (TAN) {
            float2 pp[4], dp[4], A[4], B[4], nA[4], nB[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float4 x = sc[idx[c]];
                const float4 y = sb[idx[c]];
                pp[c] = lo2(x); dp[c] = hi2(x); A[c] = lo2(y); B[c] = hi2(y);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float2 e1 = make_float2(red[2 * (i * 4 + j)], red[2 * (i * 4 + j) + 1]);
                    M::cmac(e1, A[i], pp[j], pp[j]);
                    red[2 * (i * 4 + j)] = e1.x;
                    red[2 * (i * 4 + j) + 1] = e1.y;
                    float2 e2 = make_float2(red[32 + 2 * (i * 4 + j)], red[32 + 2 * (i * 4 + j) + 1]);
                    M::cmac(e2, B[i], pp[j], pp[j]);
                    M::cmac(e2, A[i], dp[j], dp[j]);
                    red[32 + 2 * (i * 4 + j)] = e2.x;
                    red[32 + 2 * (i * 4 + j) + 1] = e2.y;
                }
            matvec4<false>(Gh, A, A, nA);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                nB[r] = make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < 4; ++c) M::mac(nB[r], Vh[r * 4 + c], A[c], A[c]);
#pragma unroll
                for (int c = 0; c < 4; ++c) M::mac(nB[r], Gh[r * 4 + c], B[c], B[c]);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) sb[idx[r]] = make_float4(nA[r].x, nA[r].y, nB[r].x, nB[r].y);
        } else {
            float2 pp[4], A[4], nA[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) { pp[c] = sc[idx[c]]; A[c] = sb[idx[c]]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float2 e1 = make_float2(red[2 * (i * 4 + j)], red[2 * (i * 4 + j) + 1]);
                    M::cmac(e1, A[i], pp[j], pp[j]);
                    red[2 * (i * 4 + j)] = e1.x;
                    red[2 * (i * 4 + j) + 1] = e1.y;
                }
            matvec4<false>(Gh, A, A, nA);
#pragma unroll
            for (int r = 0; r < 4; ++r) sb[idx[r]] = nA[r];
        }
    }
}

// Two groups per iteration (scalar arithmetic): every matrix element read from
// shared memory feeds both groups, and the two groups give independent
// instruction streams. Requires (Lt / 4) % (2 NT) == 0.
template <bool TAN, int NT, int NV>
__device__ __forceinline__ void bwd_gate2(typename Elt<TAN>::T* __restrict__ sf, typename Elt<TAN>::T* __restrict__ sb,
                                          const float2* Gi, const float2* Gh, const float2* Vm, const float2* Vh,
                                          int u, int v, int Lt, float (&red)[NV]) {
    using M = Math<false>;
    const int tid = threadIdx.x;
    const int plo = min(u, v), phi_ = max(u, v);
    const unsigned mu = 1u << u, mv = 1u << v;
    for (int q = tid; q < (Lt >> 2); q += 2 * NT) {
        unsigned idx[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const unsigned l0 = insert0(insert0(q + h * NT, plo), phi_);
            idx[h][0] = swz(l0); idx[h][1] = swz(l0 | mv); idx[h][2] = swz(l0 | mu); idx[h][3] = swz(l0 | mu | mv);
        }
        if constexpr (TAN) {
            float2 p[2][4], d[2][4], A[2][4], B[2][4];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float4 x = sf[idx[h][c]];
                    const float4 y = sb[idx[h][c]];
                    p[h][c] = lo2(x); d[h][c] = hi2(x); A[h][c] = lo2(y); B[h][c] = hi2(y);
                }
            float2 pp[2][4], dp[2][4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                pp[0][r] = pp[1][r] = make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float2 m = Gi[r * 4 + c];
                    M::mac(pp[0][r], m, p[0][c], p[0][c]);
                    M::mac(pp[1][r], m, p[1][c], p[1][c]);
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {                     // dp = G^-1 d - Y p
                dp[0][r] = dp[1][r] = make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float2 m = Gi[r * 4 + c], y = Vm[r * 4 + c];
                    M::mac(dp[0][r], m, d[0][c], d[0][c]);
                    M::mac(dp[1][r], m, d[1][c], d[1][c]);
                    M::msub(dp[0][r], y, p[0][c], p[0][c]);
                    M::msub(dp[1][r], y, p[1][c], p[1][c]);
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float2 e1 = make_float2(red[2 * (i * 4 + j)], red[2 * (i * 4 + j) + 1]);
                        M::cmac(e1, A[h][i], pp[h][j], pp[h][j]);
                        red[2 * (i * 4 + j)] = e1.x;
                        red[2 * (i * 4 + j) + 1] = e1.y;
                        float2 e2 = make_float2(red[32 + 2 * (i * 4 + j)], red[32 + 2 * (i * 4 + j) + 1]);
                        M::cmac(e2, B[h][i], pp[h][j], pp[h][j]);
                        M::cmac(e2, A[h][i], dp[h][j], dp[h][j]);
                        red[32 + 2 * (i * 4 + j)] = e2.x;
                        red[32 + 2 * (i * 4 + j) + 1] = e2.y;
                    }
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int r = 0; r < 4; ++r) sf[idx[h][r]] = make_float4(pp[h][r].x, pp[h][r].y, dp[h][r].x, dp[h][r].y);
            float2 nA[2][4], nB[2][4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                nA[0][r] = nA[1][r] = nB[0][r] = nB[1][r] = make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float2 g = Gh[r * 4 + c], vh = Vh[r * 4 + c];
                    M::mac(nA[0][r], g, A[0][c], A[0][c]);
                    M::mac(nA[1][r], g, A[1][c], A[1][c]);
                    M::mac(nB[0][r], g, B[0][c], B[0][c]);
                    M::mac(nB[1][r], g, B[1][c], B[1][c]);
                    M::mac(nB[0][r], vh, A[0][c], A[0][c]);
                    M::mac(nB[1][r], vh, A[1][c], A[1][c]);
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int r = 0; r < 4; ++r) sb[idx[h][r]] = make_float4(nA[h][r].x, nA[h][r].y, nB[h][r].x, nB[h][r].y);
        } else {
            float2 p[2][4], A[2][4], pp[2][4], nA[2][4];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int c = 0; c < 4; ++c) { p[h][c] = sf[idx[h][c]]; A[h][c] = sb[idx[h][c]]; }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                pp[0][r] = pp[1][r] = nA[0][r] = nA[1][r] = make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float2 m = Gi[r * 4 + c], g = Gh[r * 4 + c];
                    M::mac(pp[0][r], m, p[0][c], p[0][c]);
                    M::mac(pp[1][r], m, p[1][c], p[1][c]);
                    M::mac(nA[0][r], g, A[0][c], A[0][c]);
                    M::mac(nA[1][r], g, A[1][c], A[1][c]);
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float2 e1 = make_float2(red[2 * (i * 4 + j)], red[2 * (i * 4 + j) + 1]);
                        M::cmac(e1, A[h][i], pp[h][j], pp[h][j]);
                        red[2 * (i * 4 + j)] = e1.x;
                        red[2 * (i * 4 + j) + 1] = e1.y;
                    }
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int r = 0; r < 4; ++r) { sf[idx[h][r]] = pp[h][r]; sb[idx[h][r]] = nA[h][r]; }
        }
    }
}

}  // namespace tile
}  // namespace hvp
