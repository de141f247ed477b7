// Window-pass kernel of the complex64 sweep (sm_103a).
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
// Environment sums: per thread in FP32 over its groups of four amplitudes,
// a warp reduce-scatter (each lane ends with two of the 64 real components),
// a cross-warp sum in FP64 in shared memory, and one FP64 record per
// (gate, sample, CTA) in global memory.
#include <type_traits>

#include "internal.h"

namespace hvp {

namespace {

__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {  // acc += a b
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

__device__ __forceinline__ void cmac_conj(float2& acc, float2 a, float2 b) {  // acc += conj(a) b
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(-a.y, b.x, acc.y);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ unsigned insert0(unsigned x, int p) {
    return ((x >> p) << (p + 1)) | (x & ((1u << p) - 1u));
}

// y = M x for a 4x4 complex matrix in shared memory (row-major).
__device__ __forceinline__ void matvec4(const float2* __restrict__ M, const float2 (&x)[4], float2 (&y)[4]) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 4; ++c) cmac(acc, M[r * 4 + c], x[c]);
        y[r] = acc;
    }
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

}  // namespace

template <bool TAN, int NT>
__global__ void __launch_bounds__(NT, 1) tiled_pass_kernel(TiledArgs a) {
    using E = typename Elt<TAN>::T;
    constexpr int NW = NT / 32;
    constexpr int NV = TAN ? 64 : 32;          // real components of one gate's sums
    extern __shared__ __align__(16) unsigned char smem[];

    const DevPass* __restrict__ P = a.pass;
    const int w = P->w, ng = P->ng, ngates = P->n_gates, goff = P->gate_off;
    const int Lt = 1 << w;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s = blockIdx.y;
    const int mode = a.mode;
    const bool bwd = (mode & M_BWD) != 0;

    E* sf = reinterpret_cast<E*>(smem);
    E* sb = sf + Lt;
    float2* mats = reinterpret_cast<float2*>(sb + (bwd ? Lt : 0));
    float* wred = reinterpret_cast<float*>(mats + ngates * 80);
    double* acc = reinterpret_cast<double*>(wred + 2 * NW * 64);

    // Gate matrices of this pass (G, G^-1, G^dag, V, V^dag per gate).
    for (int i = tid; i < ngates * 80; i += NT) {
        const int g = i / 80, e = i - g * 80;
        const int k = __ldg(&a.gates[goff + g].k);
        mats[i] = reinterpret_cast<const float2*>(a.mats + k)[e];
    }
    if (bwd)
        for (int i = tid; i < ngates * NV; i += NT) acc[i] = 0.0;

    const size_t sample_off = (size_t)s << a.n;
    const uint32_t* offlo = P->off_lo;
    const uint32_t* offhi = P->off_hi;
    const uint16_t* ldlo = a.ld_out_tab ? P->out_lo : P->in_lo;
    const uint16_t* ldhi = a.ld_out_tab ? P->out_hi : P->in_hi;
    const uint16_t* stlo = a.st_out_tab ? P->out_lo : P->in_lo;
    const uint16_t* sthi = a.st_out_tab ? P->out_hi : P->in_hi;

    for (int it = 0; it < a.tiles_per_cta; ++it) {
        const unsigned t = blockIdx.x * a.tiles_per_cta + it;
        size_t base = sample_off;
        for (int r = 0; r < ng; ++r)
            if ((t >> r) & 1u) base |= (size_t)1 << __ldg(&P->gpos[r]);

        // ------------------------------------------------------------ load
        if (mode & M_GEN) {
            // psi^[0] = (x)_q psi_{s,q}: tile factor from the fixed qubits times
            // the factors of the window qubits (Eq. costHS, product states).
            const float2* q1 = a.psi1q + (size_t)s * a.n * 2;
            float2 gamma = make_float2(1.f, 0.f);
            for (int r = 0; r < ng; ++r) gamma = cmulf(gamma, __ldg(&q1[2 * __ldg(&P->gq[r]) + ((t >> r) & 1u)]));
            for (int l = tid; l < Lt; l += NT) {
                float2 amp = gamma;
                for (int j = 0; j < w; ++j) amp = cmulf(amp, __ldg(&q1[2 * __ldg(&P->sq[j]) + ((l >> j) & 1)]));
                if constexpr (TAN) sf[swz(l)] = make_float4(amp.x, amp.y, 0.f, 0.f);
                else sf[swz(l)] = amp;
            }
        } else {
            const E* __restrict__ xin = reinterpret_cast<const E*>(a.xin);
            for (int m = tid; m < Lt; m += NT) {
                const size_t addr = base + __ldg(&offlo[m & 63]) + __ldg(&offhi[m >> 6]);
                const unsigned l = __ldg(&ldlo[m & 63]) | __ldg(&ldhi[m >> 6]);
                sf[swz(l)] = xin[addr];
            }
        }
        if (bwd) {
            if (mode & M_LOAD_PHI) {
                for (int m = tid; m < Lt; m += NT) {
                    const size_t addr = base + __ldg(&offlo[m & 63]) + __ldg(&offhi[m >> 6]);
                    const unsigned l = __ldg(&ldlo[m & 63]) | __ldg(&ldhi[m >> 6]);
                    const float2 ph = a.phi[addr];
                    if constexpr (TAN) sb[swz(l)] = make_float4(ph.x, ph.y, 0.f, 0.f);
                    else sb[swz(l)] = ph;
                }
            } else {
                const E* __restrict__ cin = reinterpret_cast<const E*>(a.cin);
                for (int m = tid; m < Lt; m += NT) {
                    const size_t addr = base + __ldg(&offlo[m & 63]) + __ldg(&offhi[m >> 6]);
                    const unsigned l = __ldg(&ldlo[m & 63]) | __ldg(&ldhi[m >> 6]);
                    sb[swz(l)] = cin[addr];
                }
            }
        }
        __syncthreads();

        // --------------------------------------------------- forward gates
        if (mode & M_FWD) {
            for (int g = 0; g < ngates; ++g) {
                const DevGate dg = a.gates[goff + g];
                const float2* Gm = mats + g * 80;
                const float2* Vm = Gm + 48;
                const int u = dg.u, v = dg.v;
                const int plo = min(u, v), phi_ = max(u, v);
                const unsigned mu = 1u << u, mv = 1u << v;
                for (int q = tid; q < (Lt >> 2); q += NT) {
                    const unsigned l0 = insert0(insert0(q, plo), phi_);
                    const unsigned idx[4] = {swz(l0), swz(l0 | mv), swz(l0 | mu), swz(l0 | mu | mv)};
                    if constexpr (TAN) {
                        float2 p[4], d[4], np[4], nd[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) { const float4 x = sf[idx[c]]; p[c] = lo2(x); d[c] = hi2(x); }
                        matvec4(Gm, p, np);
                        matvec4(Gm, d, nd);
#pragma unroll
                        for (int r = 0; r < 4; ++r)
#pragma unroll
                            for (int c = 0; c < 4; ++c) cmac(nd[r], Vm[r * 4 + c], p[c]);
#pragma unroll
                        for (int r = 0; r < 4; ++r) sf[idx[r]] = make_float4(np[r].x, np[r].y, nd[r].x, nd[r].y);
                    } else {
                        float2 p[4], np[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) p[c] = sf[idx[c]];
                        matvec4(Gm, p, np);
#pragma unroll
                        for (int r = 0; r < 4; ++r) sf[idx[r]] = np[r];
                    }
                }
                __syncthreads();
            }
        }

        // ------------------------------------------------------ store forward
        if (mode & M_STORE_F) {
            E* __restrict__ xout = reinterpret_cast<E*>(a.xout);
            for (int m = tid; m < Lt; m += NT) {
                const size_t addr = base + __ldg(&offlo[m & 63]) + __ldg(&offhi[m >> 6]);
                const unsigned l = __ldg(&stlo[m & 63]) | __ldg(&sthi[m >> 6]);
                xout[addr] = sf[swz(l)];
            }
        }

        // -------------------------------------------------- backward gates
        if (bwd) {
            for (int g = ngates - 1; g >= 0; --g) {
                const DevGate dg = a.gates[goff + g];
                const float2* Gi = mats + g * 80 + 16;
                const float2* Gh = mats + g * 80 + 32;
                const float2* Vm = mats + g * 80 + 48;
                const float2* Vh = mats + g * 80 + 64;
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
                        float2 p[4], d[4], A[4], B[4], pp[4], tt[4], dp[4], nA[4], nB[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float4 x = sf[idx[c]];
                            const float4 y = sb[idx[c]];
                            p[c] = lo2(x); d[c] = hi2(x); A[c] = lo2(y); B[c] = hi2(y);
                        }
                        matvec4(Gi, p, pp);                       // psi^[k-1]
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            tt[r] = d[r];
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const float2 vv = Vm[r * 4 + c];
                                cmac(tt[r], make_float2(-vv.x, -vv.y), pp[c]);
                            }
                        }
                        matvec4(Gi, tt, dp);                      // dpsi^[k-1]
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                float2 e1 = make_float2(red[2 * (i * 4 + j)], red[2 * (i * 4 + j) + 1]);
                                cmac_conj(e1, A[i], pp[j]);
                                red[2 * (i * 4 + j)] = e1.x;
                                red[2 * (i * 4 + j) + 1] = e1.y;
                                float2 e2 = make_float2(red[32 + 2 * (i * 4 + j)], red[32 + 2 * (i * 4 + j) + 1]);
                                cmac_conj(e2, B[i], pp[j]);
                                cmac_conj(e2, A[i], dp[j]);
                                red[32 + 2 * (i * 4 + j)] = e2.x;
                                red[32 + 2 * (i * 4 + j) + 1] = e2.y;
                            }
                        matvec4(Gh, A, nA);
                        matvec4(Gh, B, nB);
#pragma unroll
                        for (int r = 0; r < 4; ++r)
#pragma unroll
                            for (int c = 0; c < 4; ++c) cmac(nB[r], Vh[r * 4 + c], A[c]);
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            sf[idx[r]] = make_float4(pp[r].x, pp[r].y, dp[r].x, dp[r].y);
                            sb[idx[r]] = make_float4(nA[r].x, nA[r].y, nB[r].x, nB[r].y);
                        }
                    } else {
                        float2 p[4], A[4], pp[4], nA[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) { p[c] = sf[idx[c]]; A[c] = sb[idx[c]]; }
                        matvec4(Gi, p, pp);
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                float2 e1 = make_float2(red[2 * (i * 4 + j)], red[2 * (i * 4 + j) + 1]);
                                cmac_conj(e1, A[i], pp[j]);
                                red[2 * (i * 4 + j)] = e1.x;
                                red[2 * (i * 4 + j) + 1] = e1.y;
                            }
                        matvec4(Gh, A, nA);
#pragma unroll
                        for (int r = 0; r < 4; ++r) { sf[idx[r]] = pp[r]; sb[idx[r]] = nA[r]; }
                    }
                }
                warp_reduce_scatter<NV>(red, lane);
                float* wr = wred + ((g & 1) * NW + warp) * 64;
#pragma unroll
                for (int i = 0; i < NV / 32; ++i) wr[lane * (NV / 32) + i] = red[i];
                __syncthreads();
                if (tid < NV) {
                    double sum = 0.0;
                    for (int ww = 0; ww < NW; ++ww) sum += (double)wred[((g & 1) * NW + ww) * 64 + tid];
                    acc[g * NV + tid] += sum;
                }
            }
        }

        // ------------------------------------------------- store co-states
        if (mode & M_STORE_B) {
            E* __restrict__ cout = reinterpret_cast<E*>(a.cout);
            for (int m = tid; m < Lt; m += NT) {
                const size_t addr = base + __ldg(&offlo[m & 63]) + __ldg(&offhi[m >> 6]);
                const unsigned l = __ldg(&stlo[m & 63]) | __ldg(&sthi[m >> 6]);
                cout[addr] = sb[swz(l)];
            }
        }
        __syncthreads();
    }

    // One FP64 record per (gate, sample, CTA).
    if (bwd) {
        for (int i = tid; i < ngates * 64; i += NT) {
            const int g = i >> 6, e = i & 63;
            const int k = a.gates[goff + g].k;
            double* dst = a.partial + (((size_t)k * a.n_samples + s) * a.cx_count + blockIdx.x) * 64;
            dst[e] = e < NV ? acc[g * NV + e] : 0.0;
        }
    }
}

size_t tiled_smem_bytes(bool tangent, bool bwd, int w, int threads, int max_gates) {
    const size_t elt = tangent ? 16 : 8;
    size_t b = elt << w;                       // forward states
    if (bwd) b += elt << w;                    // co-states
    b += (size_t)max_gates * 80 * 8;           // matrices
    b += 2 * (size_t)(threads / 32) * 64 * 4;  // cross-warp buffer
    if (bwd) b += (size_t)max_gates * (tangent ? 64 : 32) * 8;  // FP64 sums
    return b;
}

template <bool TAN, int NT>
static cudaError_t set_limit() {
    return cudaFuncSetAttribute(tiled_pass_kernel<TAN, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                227 * 1024);
}

cudaError_t tiled_set_smem_limits() {
    cudaError_t e;
    if ((e = set_limit<true, 128>()) != cudaSuccess) return e;
    if ((e = set_limit<true, 256>()) != cudaSuccess) return e;
    if ((e = set_limit<true, 512>()) != cudaSuccess) return e;
    if ((e = set_limit<false, 128>()) != cudaSuccess) return e;
    if ((e = set_limit<false, 256>()) != cudaSuccess) return e;
    return set_limit<false, 512>();
}

cudaError_t launch_tiled(const TiledArgs& a, bool tangent, int w, int threads, int n_gates,
                         cudaStream_t st) {
    const bool bwd = (a.mode & M_BWD) != 0;
    const size_t smem = tiled_smem_bytes(tangent, bwd, w, threads, n_gates);
    dim3 grid(a.cx_count, a.n_samples);
#define HVP_LAUNCH(T, N) tiled_pass_kernel<T, N><<<grid, N, smem, st>>>(a)
    if (tangent) {
        if (threads == 128) HVP_LAUNCH(true, 128);
        else if (threads == 256) HVP_LAUNCH(true, 256);
        else if (threads == 512) HVP_LAUNCH(true, 512);
        else return cudaErrorInvalidValue;
    } else {
        if (threads == 128) HVP_LAUNCH(false, 128);
        else if (threads == 256) HVP_LAUNCH(false, 256);
        else if (threads == 512) HVP_LAUNCH(false, 512);
        else return cudaErrorInvalidValue;
    }
#undef HVP_LAUNCH
    return cudaGetLastError();
}

}  // namespace hvp
