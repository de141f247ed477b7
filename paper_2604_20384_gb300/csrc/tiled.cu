// Window-pass kernels of the complex64 sweep (sm_103a).
//
// One CTA owns tiles of 2^w amplitudes (the w window qubits vary, the other
// n - w qubits are fixed) of one sample. It loads the tile's forward states
// (psi, dpsi) and, for backward work, the co-states (a, b) into shared memory,
// applies the pass's gates there and writes the tile back, so a pass costs one
// HBM round trip however many gates it holds.
//
//   forward gate k (Eq. fis, Eq. dfis):
//       dpsi <- G_k dpsi + V_k psi ,  psi <- G_k psi
//   backward gate k, with a = phi^[K-k] and b = dphi^[K-k] before the update
//   (Eq. environment, Eq. Dpsi, Eq. bis, Eq. dbis):
//       psi^[k-1]  = G_k^-1 psi^[k]
//       dpsi^[k-1] = G_k^-1 (dpsi^[k] - V_k psi^[k-1])
//       E_k  += sum_a conj(a_i) psi^[k-1]_j
//       DE_k += sum_a conj(b_i) psi^[k-1]_j + conj(a_i) dpsi^[k-1]_j
//       b <- G_k^dag b + V_k^dag a ,  a <- G_k^dag a
// The forward state psi^[k-1] is recomputed with G^-1 inside the pass; at pass
// boundaries it comes from the forward checkpoint, so recomputation error does
// not build up over the whole circuit.
//
// Two kernels: a forward-only kernel (small register footprint, two CTAs per
// SM) and a backward kernel (forward part of the turnaround pass included).
// Two arithmetic forms, chosen at run time: scalar FP32 FMAs, or packed
// fma.rn.f32x2 with gate matrices pre-expanded to {m.re, m.re, -m.im, m.im}
// so that one complex multiply-add is two packed FMAs.
//
// Environment sums: per thread in FP32 over its groups of four amplitudes,
// a warp reduce-scatter (each lane ends with two of the 64 real components),
// a cross-warp FP32 sum per gate into a per-CTA FP32 accumulator, and one
// FP64 record per (gate, sample, CTA) in global memory at the end.
#include "internal.h"

namespace hvp {

namespace {

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
template <bool P2>
__device__ __forceinline__ void matvec4(const typename Math<P2>::M* __restrict__ M, const float2 (&x)[4],
                                        const float2 (&xs)[4], float2 (&y)[4]) {
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

__device__ __forceinline__ size_t tile_base(const DevPass* __restrict__ P, unsigned t, size_t sample_off, int ng) {
    size_t base = sample_off;
    for (int r = 0; r < ng; ++r)
        if ((t >> r) & 1u) base |= (size_t)1 << __ldg(&P->gpos[r]);
    return base;
}

template <typename E, int NT>
__device__ __forceinline__ void load_tile(E* __restrict__ dst, const E* __restrict__ src, const TileCtx& tc,
                                          const uint16_t* lo, const uint16_t* hi, int Lt) {
    for (int m = threadIdx.x; m < Lt; m += NT) {
        const size_t addr = tc.base + __ldg(&tc.offlo[m & 63]) + __ldg(&tc.offhi[m >> 6]);
        const unsigned l = __ldg(&lo[m & 63]) | __ldg(&hi[m >> 6]);
        dst[swz(l)] = src[addr];
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
// of the window qubits (Eq. costHS, product states).
template <typename E, int NT>
__device__ __forceinline__ void gen_tile(E* __restrict__ sf, const DevPass* __restrict__ P, const float2* q1,
                                         unsigned t, int w, int ng, int Lt) {
    float2 gamma = make_float2(1.f, 0.f);
    for (int r = 0; r < ng; ++r) gamma = cmulf(gamma, __ldg(&q1[2 * __ldg(&P->gq[r]) + ((t >> r) & 1u)]));
    for (int l = threadIdx.x; l < Lt; l += NT) {
        float2 amp = gamma;
        for (int j = 0; j < w; ++j) amp = cmulf(amp, __ldg(&q1[2 * __ldg(&P->sq[j]) + ((l >> j) & 1)]));
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
template <bool TAN, bool P2, int NT>
__device__ __forceinline__ void fwd_gate(typename Elt<TAN>::T* __restrict__ sf, const typename Math<P2>::M* Gm,
                                         const typename Math<P2>::M* Vm, int u, int v, int Lt) {
    const int plo = min(u, v), phi_ = max(u, v);
    const unsigned mu = 1u << u, mv = 1u << v;
    for (int q = threadIdx.x; q < (Lt >> 2); q += NT) {
        const unsigned l0 = insert0(insert0(q, plo), phi_);
        const unsigned idx[4] = {swz(l0), swz(l0 | mv), swz(l0 | mu), swz(l0 | mu | mv)};
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
            for (int r = 0; r < 4; ++r) sf[idx[r]] = make_float4(np[r].x, np[r].y, nd[r].x, nd[r].y);
        } else {
            float2 p[4], ps[4], np[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) p[c] = sf[idx[c]];
            swaps<P2>(p, ps);
            matvec4<P2>(Gm, p, ps, np);
#pragma unroll
            for (int r = 0; r < 4; ++r) sf[idx[r]] = np[r];
        }
    }
}

}  // namespace

// ------------------------------------------------------------ forward kernel
template <bool TAN, bool P2, int NT>
__global__ void __launch_bounds__(NT, 2) tiled_fwd_kernel(TiledArgs a) {
    using E = typename Elt<TAN>::T;
    using MT = typename Math<P2>::M;
    extern __shared__ __align__(16) unsigned char smem[];
    const DevPass* __restrict__ P = a.pass;
    const int w = P->w, ng = P->ng, ngates = P->n_gates, goff = P->gate_off;
    const int Lt = 1 << w;
    const int s = blockIdx.y;
    E* sf = reinterpret_cast<E*>(smem);
    MT* mats = reinterpret_cast<MT*>(sf + Lt);
    const int which[kFwdMats] = {0, 3};   // G, V
    stage_mats<P2, NT>(mats, a, goff, ngates, kFwdMats, which);

    const size_t sample_off = (size_t)s << a.n;
    TileCtx tc{0, P->off_lo, P->off_hi};
    const uint16_t* ldlo = a.ld_out_tab ? P->out_lo : P->in_lo;
    const uint16_t* ldhi = a.ld_out_tab ? P->out_hi : P->in_hi;
    const uint16_t* stlo = a.st_out_tab ? P->out_lo : P->in_lo;
    const uint16_t* sthi = a.st_out_tab ? P->out_hi : P->in_hi;
    for (int it = 0; it < a.tiles_per_cta; ++it) {
        const unsigned t = blockIdx.x * a.tiles_per_cta + it;
        tc.base = tile_base(P, t, sample_off, ng);
        if (a.mode & M_GEN) gen_tile<E, NT>(sf, P, a.psi1q + (size_t)s * a.n * 2, t, w, ng, Lt);
        else load_tile<E, NT>(sf, reinterpret_cast<const E*>(a.xin), tc, ldlo, ldhi, Lt);
        __syncthreads();
        for (int g = 0; g < ngates; ++g) {
            const DevGate dg = a.gates[goff + g];
            fwd_gate<TAN, P2, NT>(sf, mats + (g * kFwdMats) * 16, mats + (g * kFwdMats + 1) * 16, dg.u, dg.v, Lt);
            __syncthreads();
        }
        if (a.mode & M_STORE_F) store_tile<E, NT>(reinterpret_cast<E*>(a.xout), sf, tc, stlo, sthi, Lt);
        __syncthreads();
    }
}

// ----------------------------------------------------------- backward kernel
template <bool TAN, bool P2, int NT>
__global__ void __launch_bounds__(NT, 1) tiled_bwd_kernel(TiledArgs a) {
    using E = typename Elt<TAN>::T;
    using MT = typename Math<P2>::M;
    constexpr int NW = NT / 32;
    constexpr int NV = TAN ? 64 : 32;          // real components of one gate's sums
    extern __shared__ __align__(16) unsigned char smem[];

    const DevPass* __restrict__ P = a.pass;
    const int w = P->w, ng = P->ng, ngates = P->n_gates, goff = P->gate_off;
    const int Lt = 1 << w;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s = blockIdx.y;
    const int mode = a.mode;

    const int nmat = (mode & M_FWD) ? 5 : 4;
    E* sf = reinterpret_cast<E*>(smem);
    E* sb = sf + Lt;
    MT* mats = reinterpret_cast<MT*>(sb + Lt);
    float* wred = reinterpret_cast<float*>(mats + ngates * nmat * 16);
    float* acc = wred + 2 * NW * 64;           // [ngates][NV] FP32 per CTA

    const int which[5] = {1, 2, 3, 4, 0};      // G^-1, G^dag, V, V^dag, G
    stage_mats<P2, NT>(mats, a, goff, ngates, nmat, which);
    for (int i = tid; i < ngates * NV; i += NT) acc[i] = 0.f;

    const size_t sample_off = (size_t)s << a.n;
    TileCtx tc{0, P->off_lo, P->off_hi};
    const uint16_t* ldlo = a.ld_out_tab ? P->out_lo : P->in_lo;
    const uint16_t* ldhi = a.ld_out_tab ? P->out_hi : P->in_hi;
    const uint16_t* stlo = a.st_out_tab ? P->out_lo : P->in_lo;
    const uint16_t* sthi = a.st_out_tab ? P->out_hi : P->in_hi;

    for (int it = 0; it < a.tiles_per_cta; ++it) {
        const unsigned t = blockIdx.x * a.tiles_per_cta + it;
        tc.base = tile_base(P, t, sample_off, ng);
        if (mode & M_GEN) gen_tile<E, NT>(sf, P, a.psi1q + (size_t)s * a.n * 2, t, w, ng, Lt);
        else load_tile<E, NT>(sf, reinterpret_cast<const E*>(a.xin), tc, ldlo, ldhi, Lt);
        if (mode & M_LOAD_PHI) {
            for (int m = tid; m < Lt; m += NT) {
                const size_t addr = tc.base + __ldg(&tc.offlo[m & 63]) + __ldg(&tc.offhi[m >> 6]);
                const unsigned l = __ldg(&ldlo[m & 63]) | __ldg(&ldhi[m >> 6]);
                const float2 ph = a.phi[addr];
                if constexpr (TAN) sb[swz(l)] = make_float4(ph.x, ph.y, 0.f, 0.f);
                else sb[swz(l)] = ph;
            }
        } else {
            load_tile<E, NT>(sb, reinterpret_cast<const E*>(a.cin), tc, ldlo, ldhi, Lt);
        }
        __syncthreads();

        // Turnaround pass: forward through the gates first.
        if (mode & M_FWD) {
            for (int g = 0; g < ngates; ++g) {
                const DevGate dg = a.gates[goff + g];
                fwd_gate<TAN, P2, NT>(sf, mats + (g * nmat + 4) * 16, mats + (g * nmat + 2) * 16, dg.u, dg.v, Lt);
                __syncthreads();
            }
        }

        for (int g = ngates - 1; g >= 0; --g) {
            const DevGate dg = a.gates[goff + g];
            const MT* Gi = mats + (g * nmat + 0) * 16;
            const MT* Gh = mats + (g * nmat + 1) * 16;
            const MT* Vm = mats + (g * nmat + 2) * 16;
            const MT* Vh = mats + (g * nmat + 3) * 16;
            const int u = dg.u, v = dg.v;
            const int plo = min(u, v), phi_ = max(u, v);
            const unsigned mu = 1u << u, mv = 1u << v;
            float red[NV];
#pragma unroll
            for (int e = 0; e < NV; ++e) red[e] = 0.f;
            for (int q = tid; q < (Lt >> 2); q += NT) {
                const unsigned l0 = insert0(insert0(q, plo), phi_);
                const unsigned idx[4] = {swz(l0), swz(l0 | mv), swz(l0 | mu), swz(l0 | mu | mv)};
                if constexpr (TAN) {
                    float2 p[4], d[4], A[4], B[4], xs[4], pp[4], pps[4], tt[4], dp[4], dps[4], nA[4], nB[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float4 x = sf[idx[c]];
                        const float4 y = sb[idx[c]];
                        p[c] = lo2(x); d[c] = hi2(x); A[c] = lo2(y); B[c] = hi2(y);
                    }
                    swaps<P2>(p, xs);
                    matvec4<P2>(Gi, p, xs, pp);                       // psi^[k-1]
                    swaps<P2>(pp, pps);
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        tt[r] = d[r];
#pragma unroll
                        for (int c = 0; c < 4; ++c) Math<P2>::msub(tt[r], Vm[r * 4 + c], pp[c], pps[c]);
                    }
                    swaps<P2>(tt, xs);
                    matvec4<P2>(Gi, tt, xs, dp);                      // dpsi^[k-1]
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
            warp_reduce_scatter<NV>(red, lane);
            float* wr = wred + ((g & 1) * NW + warp) * 64;
#pragma unroll
            for (int i = 0; i < NV / 32; ++i) wr[lane * (NV / 32) + i] = red[i];
            __syncthreads();
            // Cross-warp sum of this gate in FP32, spread over NV threads; the
            // double-buffered slot (gate parity) is rewritten two gates later.
            if (tid < NV) {
                float sum = 0.f;
#pragma unroll
                for (int ww = 0; ww < NW; ++ww) sum += wred[((g & 1) * NW + ww) * 64 + tid];
                acc[g * NV + tid] += sum;
            }
        }

        if (mode & M_STORE_B) store_tile<E, NT>(reinterpret_cast<E*>(a.cout), sb, tc, stlo, sthi, Lt);
        __syncthreads();
    }

    // One FP64 record per (gate, sample, CTA).
    for (int i = tid; i < ngates * 64; i += NT) {
        const int g = i >> 6, e = i & 63;
        const int k = a.gates[goff + g].k;
        double* dst = a.partial + (((size_t)k * a.n_samples + s) * a.cx_count + blockIdx.x) * 64;
        dst[e] = e < NV ? (double)acc[g * NV + e] : 0.0;
    }
}

size_t tiled_smem_bytes(bool tangent, int mode, int w, int threads, int max_gates, int variant) {
    const bool bwd = (mode & M_BWD) != 0;
    const size_t elt = tangent ? 16 : 8;
    const size_t mb = variant == 2 ? 16 : 8;
    size_t b = elt << w;                                       // forward states
    if (bwd) {
        b += elt << w;                                         // co-states
        b += (size_t)max_gates * ((mode & M_FWD) ? 5 : 4) * 16 * mb;   // matrices
        b += 2 * (size_t)(threads / 32) * 64 * 4;              // cross-warp buffer
        b += (size_t)max_gates * (tangent ? 64 : 32) * 4;      // FP32 sums
    } else {
        b += (size_t)max_gates * kFwdMats * 16 * mb;
    }
    return b;
}

template <bool TAN, bool P2, int NT>
static cudaError_t set_limits_one() {
    cudaError_t e = cudaFuncSetAttribute(tiled_fwd_kernel<TAN, P2, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(tiled_bwd_kernel<TAN, P2, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                227 * 1024);
}

cudaError_t tiled_set_smem_limits() {
    cudaError_t e;
#define HVP_SET(T, P, N) if ((e = set_limits_one<T, P, N>()) != cudaSuccess) return e
    HVP_SET(true, false, 256); HVP_SET(true, false, 512); HVP_SET(true, true, 256); HVP_SET(true, true, 512);
    HVP_SET(false, false, 256); HVP_SET(false, false, 512); HVP_SET(false, true, 256); HVP_SET(false, true, 512);
#undef HVP_SET
    return cudaSuccess;
}

cudaError_t launch_tiled(const TiledArgs& a, bool tangent, int w, int threads, int n_gates, cudaStream_t st,
                         int variant) {
    const bool bwd = (a.mode & M_BWD) != 0;
    const bool p2 = variant == 2;
    const size_t smem = tiled_smem_bytes(tangent, a.mode, w, threads, n_gates, variant);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    dim3 grid(a.cx_count, a.n_samples);
#define HVP_L(K, T, P, N) K<T, P, N><<<grid, N, smem, st>>>(a)
#define HVP_PICK(K)                                                                                  \
    if (tangent) {                                                                                   \
        if (p2) { if (threads == 512) HVP_L(K, true, true, 512); else HVP_L(K, true, true, 256); }    \
        else { if (threads == 512) HVP_L(K, true, false, 512); else HVP_L(K, true, false, 256); }     \
    } else {                                                                                         \
        if (p2) { if (threads == 512) HVP_L(K, false, true, 512); else HVP_L(K, false, true, 256); }  \
        else { if (threads == 512) HVP_L(K, false, false, 512); else HVP_L(K, false, false, 256); }   \
    }
    if (threads != 256 && threads != 512) return cudaErrorInvalidValue;
    if (bwd) {
        HVP_PICK(tiled_bwd_kernel)
    } else {
        HVP_PICK(tiled_fwd_kernel)
    }
#undef HVP_PICK
#undef HVP_L
    return cudaGetLastError();
}

}  // namespace hvp
