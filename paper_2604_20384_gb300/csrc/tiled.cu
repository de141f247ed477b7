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
//       dpsi^[k-1] = G_k^-1 dpsi^[k] - Y_k psi^[k],  Y_k = G_k^-1 V_k G_k^-1
//                    (= G_k^-1 (dpsi^[k] - V_k psi^[k-1]))
//       E_k  += sum_a conj(a_i) psi^[k-1]_j
//       DE_k += sum_a conj(b_i) psi^[k-1]_j + conj(a_i) dpsi^[k-1]_j
//       b <- G_k^dag b + V_k^dag a ,  a <- G_k^dag a
// Recompute schedule: the forward state psi^[k-1] is recomputed with G^-1
// inside the pass; at pass boundaries it comes from the forward checkpoint,
// so recomputation error does not build up over the whole circuit. Forward-
// cache schedule: psi^[k-1], dpsi^[k-1] are read from the cache.
//
// Kernels: a forward kernel (small register footprint: two CTAs per SM at
// 256 threads, four at 128), optionally writing the forward cache (the
// states before every gate, as Alg. 1 keeps them); a recomputing backward
// kernel (forward part of the turnaround pass included; 255 registers: one
// CTA per SM at 256 threads, two at 128); and a backward kernel that reads
// the forward cache by bulk copies instead of recomputing (tiled_bwdc_kernel,
// 24 instead of 36 complex multiply-adds per amplitude per gate).
// Arithmetic forms of the recompute schedule, chosen at run time: scalar
// FP32 FMAs (variant 1), packed fma.rn.f32x2 with gate matrices pre-expanded
// to {m.re, m.re, -m.im, m.im} so that one complex multiply-add is two packed
// FMAs (variant 2), or scalar with two groups per thread iteration in the
// backward pass (variant 3).
//
// Environment sums: per thread in FP32 over its groups of four amplitudes,
// a warp reduce-scatter (each lane ends with two of the 64 real components),
// a cross-warp FP32 sum per gate into a per-CTA FP32 accumulator, and one
// FP64 record per (gate, sample, CTA) in global memory at the end.
#include "tiled_common.cuh"

namespace hvp {

using namespace tile;

// ------------------------------------------------------------ forward kernel
template <bool TAN, bool P2, int NT, int GPT = 0, bool DUMP = false>
__global__ void __launch_bounds__(NT, NT <= 128 ? 4 : 2) tiled_fwd_kernel(TiledArgs a) {
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
        if (a.mode & M_GEN) gen_tile<E, NT>(sf, P, a.psi1q + (size_t)s * a.n * 2, t, P->nq, ng, Lt, a.n);
        else load_tile<E, NT>(sf, reinterpret_cast<const E*>(a.xin), tc, ldlo, ldhi, Lt);
        __syncthreads();
        if (DUMP && ngates > 0) {   // forward cache: the states before the pass's first gate
            E* d0 = cache_tile<E>(a, goff, s, t, P->ng, Lt);
            for (int m = threadIdx.x; m < Lt; m += NT) d0[m] = sf[m];
            __syncthreads();         // the first gate updates the tile in place
        }
        for (int g = 0; g < ngates; ++g) {
            const DevGate dg = a.gates[goff + g];
            const MT* Gm = mats + (g * kFwdMats) * 16;
            const MT* Vm = mats + (g * kFwdMats + 1) * 16;
            if (DUMP && g + 1 < ngates)   // and the states after every gate but the last
                fwd_gate<TAN, P2, NT, const MT*, GPT, true>(sf, Gm, Vm, dg.u, dg.v, Lt,
                                                            cache_tile<E>(a, goff + g + 1, s, t, P->ng, Lt));
            else
                fwd_gate<TAN, P2, NT, const MT*, GPT>(sf, Gm, Vm, dg.u, dg.v, Lt);
            __syncthreads();
        }
        if (a.mode & M_STORE_F) store_tile<E, NT>(reinterpret_cast<E*>(a.xout), sf, tc, stlo, sthi, Lt);
        __syncthreads();
    }
}

// ----------------------------------------------------------- backward kernel
template <bool TAN, bool P2, int NT, bool G2 = false, int GPT = 0>
__global__ void __launch_bounds__(NT, NT <= 128 ? 2 : 1) tiled_bwd_kernel(TiledArgs a) {
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

    const int nmat = (mode & M_FWD) ? 6 : 4;
    E* sf = reinterpret_cast<E*>(smem);
    E* sb = sf + Lt;
    MT* mats = reinterpret_cast<MT*>(sb + Lt);
    float* wred = reinterpret_cast<float*>(mats + ngates * nmat * 16);
    float* acc = wred + 2 * NW * 64;           // [ngates][NV] FP32 per CTA

    const int which[6] = {1, 2, 5, 4, 0, 3};   // G^-1, G^dag, Y, V^dag, G, V
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
        if (mode & M_GEN) gen_tile<E, NT>(sf, P, a.psi1q + (size_t)s * a.n * 2, t, P->nq, ng, Lt, a.n);
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
                fwd_gate<TAN, P2, NT, const MT*, GPT>(sf, mats + (g * nmat + 4) * 16, mats + (g * nmat + 5) * 16, dg.u,
                                                       dg.v, Lt);
                __syncthreads();
            }
        }

        for (int g = ngates - 1; g >= 0; --g) {
            const DevGate dg = a.gates[goff + g];
            const MT* Gi = mats + (g * nmat + 0) * 16;
            const MT* Gh = mats + (g * nmat + 1) * 16;
            const MT* Vm = mats + (g * nmat + 2) * 16;
            const MT* Vh = mats + (g * nmat + 3) * 16;
            float red[NV];
#pragma unroll
            for (int e = 0; e < NV; ++e) red[e] = 0.f;
            if constexpr (G2 && !P2) {
                if (((Lt >> 2) % (2 * NT)) == 0) bwd_gate2<TAN, NT, NV>(sf, sb, Gi, Gh, Vm, Vh, dg.u, dg.v, Lt, red);
                else bwd_gate<TAN, false, NT, NV>(sf, sb, Gi, Gh, Vm, Vh, dg.u, dg.v, Lt, red);
            } else {
                bwd_gate<TAN, P2, NT, NV, const MT*, GPT>(sf, sb, Gi, Gh, Vm, Vh, dg.u, dg.v, Lt, red);
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

// ------------------------------------------- backward kernel, cached states
// Forward states before every gate are read from the forward cache instead of
// being recomputed with G^-1: per gate, the tile's cached states (one
// contiguous 2^w-element block in shared-memory order) arrive by a bulk copy
// into one of two shared-memory buffers while the previous gate is computed.
// Thread 0 issues the copies; every thread waits on the copy's mbarrier with
// a bound. A thread that gives up raises a shared stop flag and bit 2 of
// *a.status; the flag is read after a barrier, so the CTA leaves its loops
// together, thread 0 waits (again bounded) for its copies in flight, and the
// CTA returns without writing environment records.
constexpr unsigned kCopyWaitLimit = 1u << 23;

template <bool TAN, int NT, int GPT = 0>
__global__ void __launch_bounds__(NT, 1) tiled_bwdc_kernel(TiledArgs a) {
    using E = typename Elt<TAN>::T;
    constexpr int NW = NT / 32;
    constexpr int NV = TAN ? 64 : 32;
    extern __shared__ __align__(128) unsigned char smem[];

    const DevPass* __restrict__ P = a.pass;
    const int w = P->w, ng = P->ng, ngates = P->n_gates, goff = P->gate_off;
    const int Lt = 1 << w;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s = blockIdx.y;
    const int mode = a.mode;
    const unsigned bytes = (unsigned)(Lt * sizeof(E));
    const unsigned wait_limit = a.copy_wait_limit ? a.copy_wait_limit : kCopyWaitLimit;
    const unsigned extra = a.copy_extra_bytes;

    E* sb = reinterpret_cast<E*>(smem);
    E* const buf0 = sb + Lt;       // cache buffers (even and odd steps of the gate loop)
    E* const buf1 = sb + 2 * Lt;
    float2* mats = reinterpret_cast<float2*>(sb + 3 * Lt);     // [gate][G^dag, V^dag][16]
    float* wred = reinterpret_cast<float*>(mats + ngates * 2 * 16);
    float* acc = wred + 2 * NW * 64;                           // [ngates][NV] FP32 per CTA
    uint64_t* bars = reinterpret_cast<uint64_t*>(acc + ngates * NV);
    volatile int* stop = reinterpret_cast<volatile int*>(bars + 2);   // [step parity]
    int2* guv = reinterpret_cast<int2*>(bars + 3);            // [gate] shared-memory bits (u, v)

    const int which[2] = {2, 4};   // G^dag, V^dag
    stage_mats<false, NT>(mats, a, goff, ngates, 2, which);
    for (int i = tid; i < ngates; i += NT) guv[i] = make_int2(a.gates[goff + i].u, a.gates[goff + i].v);
    for (int i = tid; i < ngates * NV; i += NT) acc[i] = 0.f;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        stop[0] = 0;
        stop[1] = 0;
        fence_barrier_init();
    }
    __syncthreads();

    // Copy bookkeeping, one bit per buffer: parity of the barrier's next phase
    // (every thread), and whether a copy into the buffer is outstanding
    // (thread 0, which issues them).
    unsigned par = 0u, pend = 0u;
    const size_t sample_off = (size_t)s << a.n;
    TileCtx tc{0, P->off_lo, P->off_hi};
    const uint16_t* ldlo = a.ld_out_tab ? P->out_lo : P->in_lo;
    const uint16_t* ldhi = a.ld_out_tab ? P->out_hi : P->in_hi;
    const uint16_t* stlo = a.st_out_tab ? P->out_lo : P->in_lo;
    const uint16_t* sthi = a.st_out_tab ? P->out_hi : P->in_hi;

    for (int it = 0; it < a.tiles_per_cta; ++it) {
        const unsigned t = blockIdx.x * a.tiles_per_cta + it;
        tc.base = tile_base(P, t, sample_off, ng);
        if (tid == 0 && ngates > 0) {   // cached states of the pass's last two gates
            fence_proxy_async_smem();
            bulk_load_async(buf0, cache_tile<E>(a, goff + ngates - 1, s, t, ng, Lt), bytes, &bars[0], extra);
            pend |= 1u;
            if (ngates > 1) {
                bulk_load_async(buf1, cache_tile<E>(a, goff + ngates - 2, s, t, ng, Lt), bytes, &bars[1], extra);
                pend |= 2u;
            }
        }
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
        __syncthreads();   // the tile's co-states are in place before any warp starts a gate

        // One barrier per gate. Every thread waits for the cached states itself;
        // a thread whose wait expires raises the stop flag of this step's parity
        // and goes on with the stale buffer (its reads stay in bounds). The flag
        // is read after the barrier that ends the step: only this step's waits
        // can have set it (a wait of step i + 2 starts after the barrier of step
        // i + 1), so every thread leaves at the same step.
        for (int i = 0; i < ngates; ++i) {
            const int g = ngates - 1 - i, b = i & 1;
            E* const cur = b ? buf1 : buf0;
            if (mbar_wait_bounded(&bars[b], (par >> b) & 1u, wait_limit)) {
                par ^= 1u << b;
                pend &= ~(1u << b);
            } else {
                stop[b] = 1;
                atomicOr(a.status, 2);
            }
            const int2 uv = guv[g];
            float red[NV];
#pragma unroll
            for (int e = 0; e < NV; ++e) red[e] = 0.f;
            bwd_gate_cached<TAN, NT, NV, GPT>(cur, sb, mats + (g * 2) * 16, mats + (g * 2 + 1) * 16, uv.x, uv.y,
                                              Lt, red);
            warp_reduce_scatter<NV>(red, lane);
            float* wr = wred + ((g & 1) * NW + warp) * 64;
#pragma unroll
            for (int k = 0; k < NV / 32; ++k) wr[lane * (NV / 32) + k] = red[k];
            __syncthreads();
            if (stop[b]) break;
            if (tid == 0 && i + 2 < ngates) {   // buffer b is free again: cached states two gates ahead
                fence_proxy_async_smem();
                bulk_load_async(cur, cache_tile<E>(a, goff + g - 2, s, t, ng, Lt), bytes, &bars[b], extra);
                pend |= 1u << b;
            }
            if (tid < NV) {
                float sum = 0.f;
#pragma unroll
                for (int ww = 0; ww < NW; ++ww) sum += wred[((g & 1) * NW + ww) * 64 + tid];
                acc[g * NV + tid] += sum;
            }
        }
        if (stop[0] | stop[1]) break;
        if (mode & M_STORE_B) store_tile<E, NT>(reinterpret_cast<E*>(a.cout), sb, tc, stlo, sthi, Lt);
        __syncthreads();
    }

    if (stop[0] | stop[1]) {   // a copy did not arrive: let the ones still in flight land before the CTA ends
        if (tid == 0)
            for (int j = 0; j < 2; ++j)
                if ((pend >> j) & 1u) mbar_wait_bounded(&bars[j], (par >> j) & 1u, wait_limit);
        return;
    }
    for (int i = tid; i < ngates * 64; i += NT) {
        const int g = i >> 6, e = i & 63;
        const int k = a.gates[goff + g].k;
        double* dst = a.partial + (((size_t)k * a.n_samples + s) * a.cx_count + blockIdx.x) * 64;
        dst[e] = e < NV ? (double)acc[g * NV + e] : 0.0;
    }
}

size_t tiled_cached_smem_bytes(bool tangent, int w, int threads, int max_gates) {
    const size_t elt = tangent ? 16 : 8;
    size_t b = 3 * (elt << w);                                  // co-states + two cache buffers
    b += (size_t)max_gates * 2 * 16 * 8;                        // G^dag, V^dag
    b += 2 * (size_t)(threads / 32) * 64 * 4;                   // cross-warp buffer
    b += (size_t)max_gates * (tangent ? 64 : 32) * 4;           // FP32 sums
    b += 32 + (size_t)max_gates * 8;                            // mbarriers, stop flag, gate bits
    return b;
}

// Forward pass that also fills the forward cache (states before each gate),
// and the cached backward pass.
cudaError_t launch_tiled_cached(const TiledArgs& a, bool tangent, int w, int threads, int n_gates, cudaStream_t st) {
    const bool bwd = (a.mode & M_BWD) != 0;
    if ((a.mode & M_FWD) && bwd) return cudaErrorInvalidValue;
    if (threads != 128 && threads != 256) return cudaErrorInvalidValue;
    const size_t smem = bwd ? tiled_cached_smem_bytes(tangent, w, threads, n_gates)
                            : tiled_smem_bytes(tangent, a.mode, w, threads, n_gates, 1);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    dim3 grid(a.cx_count, a.n_samples);
    const bool gpt4 = threads == 256 && ((1 << w) >> 2) == 4 * threads;
#define HVP_C(T, N, G)                                                                            \
    do {                                                                                          \
        if (bwd) tiled_bwdc_kernel<T, N, G><<<grid, N, smem, st>>>(a);                            \
        else tiled_fwd_kernel<T, false, N, G, true><<<grid, N, smem, st>>>(a);                    \
    } while (0)
    if (gpt4) {
        if (tangent) HVP_C(true, 256, 4); else HVP_C(false, 256, 4);
    } else if (threads == 256) {
        if (tangent) HVP_C(true, 256, 0); else HVP_C(false, 256, 0);
    } else {
        if (tangent) HVP_C(true, 128, 0); else HVP_C(false, 128, 0);
    }
#undef HVP_C
    return cudaGetLastError();
}

size_t tiled_smem_bytes(bool tangent, int mode, int w, int threads, int max_gates, int variant) {
    const bool bwd = (mode & M_BWD) != 0;
    const size_t elt = tangent ? 16 : 8;
    const size_t mb = variant == 2 ? 16 : 8;   // packed form stores 16-byte matrix elements
    size_t b = elt << w;                                       // forward states
    if (bwd) {
        b += elt << w;                                         // co-states
        b += (size_t)max_gates * ((mode & M_FWD) ? 6 : 4) * 16 * mb;   // matrices
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
    e = cudaFuncSetAttribute(tiled_bwd_kernel<TAN, P2, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess || P2) return e;
    return cudaFuncSetAttribute(tiled_bwd_kernel<TAN, false, NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                227 * 1024);
}

cudaError_t tiled_set_smem_limits() {
    cudaError_t e;
#define HVP_SET(T, P, N) if ((e = set_limits_one<T, P, N>()) != cudaSuccess) return e
    HVP_SET(true, false, 256); HVP_SET(true, false, 512); HVP_SET(true, true, 256); HVP_SET(true, true, 512);
    HVP_SET(false, false, 256); HVP_SET(false, false, 512); HVP_SET(false, true, 256); HVP_SET(false, true, 512);
    HVP_SET(true, false, 128); HVP_SET(false, false, 128);
#undef HVP_SET
#define HVP_SET4(K, T, N)                                                                                  \
    if ((e = cudaFuncSetAttribute(K<T, false, N, false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                  227 * 1024)) != cudaSuccess)                                             \
        return e
    HVP_SET4(tiled_bwd_kernel, true, 256); HVP_SET4(tiled_bwd_kernel, false, 256);
#undef HVP_SET4
#define HVP_SET4(T, N)                                                                                     \
    if ((e = cudaFuncSetAttribute(tiled_fwd_kernel<T, false, N, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  227 * 1024)) != cudaSuccess)                                             \
        return e
    HVP_SET4(true, 256); HVP_SET4(false, 256);
#undef HVP_SET4
#define HVP_SETC(T, N, G)                                                                                  \
    if ((e = cudaFuncSetAttribute(tiled_bwdc_kernel<T, N, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                  227 * 1024)) != cudaSuccess ||                                           \
        (e = cudaFuncSetAttribute(tiled_fwd_kernel<T, false, N, G, true>,                                 \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024)) != cudaSuccess) \
        return e
    HVP_SETC(true, 256, 4); HVP_SETC(false, 256, 4); HVP_SETC(true, 256, 0); HVP_SETC(false, 256, 0);
    HVP_SETC(true, 128, 0); HVP_SETC(false, 128, 0);
#undef HVP_SETC
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
    if (threads == 128) {                                                                            \
        if (tangent) HVP_L(K, true, false, 128); else HVP_L(K, false, false, 128);                   \
    } else if (tangent) {                                                                            \
        if (p2) { if (threads == 512) HVP_L(K, true, true, 512); else HVP_L(K, true, true, 256); }    \
        else { if (threads == 512) HVP_L(K, true, false, 512); else HVP_L(K, true, false, 256); }     \
    } else {                                                                                         \
        if (p2) { if (threads == 512) HVP_L(K, false, true, 512); else HVP_L(K, false, true, 256); }  \
        else { if (threads == 512) HVP_L(K, false, false, 512); else HVP_L(K, false, false, 256); }   \
    }
    if (threads != 128 && threads != 256 && threads != 512) return cudaErrorInvalidValue;
    if (threads == 128 && variant != 1) return cudaErrorInvalidValue;
    // Four groups per thread at 256 threads (12-qubit tiles): kernels with the
    // group loop unrolled at compile time (3.5-4 % faster on GB300; the same
    // unrolling at 128 threads with 11-qubit tiles measured 2 % slower, so
    // that configuration keeps the loop).
    const bool gpt4 = variant == 1 && threads == 256 && ((1 << w) >> 2) == 4 * threads;
    if (gpt4) {
        if (bwd) {
            if (tangent) tiled_bwd_kernel<true, false, 256, false, 4><<<grid, 256, smem, st>>>(a);
            else tiled_bwd_kernel<false, false, 256, false, 4><<<grid, 256, smem, st>>>(a);
        } else {
            if (tangent) tiled_fwd_kernel<true, false, 256, 4><<<grid, 256, smem, st>>>(a);
            else tiled_fwd_kernel<false, false, 256, 4><<<grid, 256, smem, st>>>(a);
        }
    } else if (bwd && variant == 3) {
        if (tangent) {
            if (threads == 512) tiled_bwd_kernel<true, false, 512, true><<<grid, 512, smem, st>>>(a);
            else tiled_bwd_kernel<true, false, 256, true><<<grid, 256, smem, st>>>(a);
        } else {
            if (threads == 512) tiled_bwd_kernel<false, false, 512, true><<<grid, 512, smem, st>>>(a);
            else tiled_bwd_kernel<false, false, 256, true><<<grid, 256, smem, st>>>(a);
        }
    } else if (bwd) {
        HVP_PICK(tiled_bwd_kernel)
    } else {
        HVP_PICK(tiled_fwd_kernel)
    }
#undef HVP_PICK
#undef HVP_L
    return cudaGetLastError();
}

}  // namespace hvp
