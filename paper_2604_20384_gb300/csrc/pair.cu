// Two tangent directions per sweep (forward-cache schedule): the states psi,
// the co-states phi and the environments E are shared between two directions
// V1, V2 at the same gates G; each direction adds its own tangent states and
// DE sums. Per amplitude and gate:
//   forward  (Eq. fis, Eq. dfis):  psi <- G psi, dpsi_b <- G dpsi_b + V_b psi
//   backward (Eq. environment, Eq. Dpsi, Eq. bis, Eq. dbis), with the forward
//   states before the gate from the cache and a = phi, b_b = dphi_b before
//   the update:
//       E    += conj(a) (x) psi
//       DE_b += conj(b_b) (x) psi + conj(a) (x) dpsi_b
//       b_b  <- G^dag b_b + V_b^dag a ,  a <- G^dag a
// 20 + 40 complex multiply-adds per amplitude per gate for both directions,
// against 12 + 24 each with one direction per sweep; the cache holds
// (psi, dpsi_1, dpsi_2): 24 bytes per amplitude per gate instead of 2 x 16.
//
// Layouts. Shared memory: a float4 array (psi, dpsi_1) and a float2 array
// dpsi_2 (co-states: (phi, dphi_1) and dphi_2), both indexed by the swizzled
// tile index. Global state buffers of A amplitudes: [A float4 | A float2].
// A cache slot holds per (sample, tile) one block [2^w float4 | 2^w float2]
// in shared-memory order, so one bulk copy fills both shared arrays.
// Records: direction 1 writes (E, DE_1) to a.partial, direction 2 (E, DE_2)
// to a.partial2, each [K][N_s][CX][64], so the FP64 post-processing of the
// one-direction path runs unchanged per direction.
#include "tiled_common.cuh"

namespace hvp {

using namespace tile;

namespace {

constexpr unsigned kPairWaitLimit = 1u << 23;

// Block of tile t of sample s in cache slot `slot`.
__device__ __forceinline__ unsigned char* pair_cache_block(const TiledArgs& a, int slot, int s, unsigned t, int ng,
                                                          int Lt) {
    return static_cast<unsigned char*>(a.cache) + (size_t)slot * a.cache_slot_bytes +
           (((size_t)s << ng) + t) * (size_t)Lt * 24;
}

// Gate matrices: field f of direction 1 (slot 0, 1) and direction 2 (slot 2).
__device__ __forceinline__ void stage_pair_mats(float2* __restrict__ dst, const TiledArgs& a, int goff, int ngates,
                                                int f0, int f1) {
    for (int i = threadIdx.x; i < ngates * 48; i += blockDim.x) {
        const int g = i / 48, mi = (i / 16) % 3, e = i & 15;
        const int k = __ldg(&a.gates[goff + g].k);
        const Mats32* m = mi == 2 ? a.mats2 + k : a.mats + k;
        const int field = mi == 0 ? f0 : f1;
        dst[i] = reinterpret_cast<const float2*>(m)[field * 16 + e];
    }
}

template <int NT>
__device__ __forceinline__ void pair_load(float4* __restrict__ s4, float2* __restrict__ s2, const void* src, size_t A,
                                          const TileCtx& tc, const uint16_t* lo, const uint16_t* hi, int Lt) {
    const float4* g4 = static_cast<const float4*>(src);
    const float2* g2 = reinterpret_cast<const float2*>(g4 + A);
    for (int m = threadIdx.x; m < Lt; m += NT) {
        const size_t addr = tc.base + __ldg(&tc.offlo[m & 63]) + __ldg(&tc.offhi[m >> 6]);
        const unsigned l = swz(__ldg(&lo[m & 63]) | __ldg(&hi[m >> 6]));
        s4[l] = g4[addr];
        s2[l] = g2[addr];
    }
}

template <int NT>
__device__ __forceinline__ void pair_store(void* dst, size_t A, const float4* __restrict__ s4,
                                           const float2* __restrict__ s2, const TileCtx& tc, const uint16_t* lo,
                                           const uint16_t* hi, int Lt) {
    float4* g4 = static_cast<float4*>(dst);
    float2* g2 = reinterpret_cast<float2*>(g4 + A);
    for (int m = threadIdx.x; m < Lt; m += NT) {
        const size_t addr = tc.base + __ldg(&tc.offlo[m & 63]) + __ldg(&tc.offhi[m >> 6]);
        const unsigned l = swz(__ldg(&lo[m & 63]) | __ldg(&hi[m >> 6]));
        g4[addr] = s4[l];
        g2[addr] = s2[l];
    }
}

// ------------------------------------------------------------ forward kernel
// Forward pass for two directions that also writes the cache (the states
// before each gate).
template <int NT>
__global__ void __launch_bounds__(NT, 2) pair_fwd_kernel(TiledArgs a) {
    using M = Math<false>;
    extern __shared__ __align__(16) unsigned char smem[];
    const DevPass* __restrict__ P = a.pass;
    const int w = P->w, ng = P->ng, ngates = P->n_gates, goff = P->gate_off;
    const int Lt = 1 << w;
    const int s = blockIdx.y;
    const size_t A = (size_t)a.n_samples << a.n;
    float4* s4 = reinterpret_cast<float4*>(smem);
    float2* s2 = reinterpret_cast<float2*>(s4 + Lt);
    float2* mats = s2 + Lt;                    // [gate][G, V1, V2][16]
    stage_pair_mats(mats, a, goff, ngates, 0, 3);

    const size_t sample_off = (size_t)s << a.n;
    TileCtx tc{0, P->off_lo, P->off_hi};
    for (int it = 0; it < a.tiles_per_cta; ++it) {
        const unsigned t = blockIdx.x * a.tiles_per_cta + it;
        tc.base = tile_base(P, t, sample_off, ng);
        if (a.mode & M_GEN) {
            gen_tile<float4, NT>(s4, P, a.psi1q + (size_t)s * a.n * 2, t, P->nq, ng, Lt, a.n);
            for (int l = threadIdx.x; l < Lt; l += NT) s2[l] = make_float2(0.f, 0.f);
        } else {
            pair_load<NT>(s4, s2, a.xin, A, tc, P->in_lo, P->in_hi, Lt);
        }
        __syncthreads();
        if (ngates > 0) {   // the states before the pass's first gate
            unsigned char* blk = pair_cache_block(a, goff, s, t, ng, Lt);
            float4* d4 = reinterpret_cast<float4*>(blk);
            float2* d2 = reinterpret_cast<float2*>(d4 + Lt);
            for (int m = threadIdx.x; m < Lt; m += NT) {
                d4[m] = s4[m];
                d2[m] = s2[m];
            }
            __syncthreads();   // the first gate updates the tile in place
        }
        for (int g = 0; g < ngates; ++g) {
            const DevGate dg = a.gates[goff + g];
            const float2* Gm = mats + (g * 3) * 16;
            const float2* V1 = Gm + 16;
            const float2* V2 = Gm + 32;
            float4* d4 = nullptr;
            float2* d2 = nullptr;
            if (g + 1 < ngates) {   // the states after this gate are the next gate's input
                unsigned char* blk = pair_cache_block(a, goff + g + 1, s, t, ng, Lt);
                d4 = reinterpret_cast<float4*>(blk);
                d2 = reinterpret_cast<float2*>(d4 + Lt);
            }
            const int u = dg.u, v = dg.v, plo = min(u, v), phi_ = max(u, v);
            const unsigned mu = 1u << u, mv = 1u << v;
            for (int q = threadIdx.x; q < (Lt >> 2); q += NT) {
                const unsigned l0 = insert0(insert0(q, plo), phi_);
                const unsigned idx[4] = {swz(l0), swz(l0 | mv), swz(l0 | mu), swz(l0 | mu | mv)};
                float2 p[4], e1[4], e2[4], np[4], n1[4], n2[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float4 x = s4[idx[c]];
                    p[c] = lo2(x);
                    e1[c] = hi2(x);
                    e2[c] = s2[idx[c]];
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    np[r] = n1[r] = n2[r] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float2 gm = Gm[r * 4 + c];
                        M::mac(np[r], gm, p[c], p[c]);
                        M::mac(n1[r], gm, e1[c], e1[c]);
                        M::mac(n2[r], gm, e2[c], e2[c]);
                        M::mac(n1[r], V1[r * 4 + c], p[c], p[c]);
                        M::mac(n2[r], V2[r * 4 + c], p[c], p[c]);
                    }
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float4 o = make_float4(np[r].x, np[r].y, n1[r].x, n1[r].y);
                    s4[idx[r]] = o;
                    s2[idx[r]] = n2[r];
                    if (d4) {
                        d4[idx[r]] = o;
                        d2[idx[r]] = n2[r];
                    }
                }
            }
            __syncthreads();
        }
        if (a.mode & M_STORE_F) pair_store<NT>(a.xout, A, s4, s2, tc, P->out_lo, P->out_hi, Lt);
        __syncthreads();
    }
}

// ----------------------------------------------------------- backward kernel
// Backward pass for two directions from the cache: per gate one bulk copy of
// the tile's cached block into one of two shared-memory buffers, one gate
// ahead, with bounded mbarrier waits (as in the one-direction kernel: an
// expired wait sets bit 2 of *a.status, the CTA stops together, waits
// bounded for its copies in flight and writes no records).
template <int NT>
__global__ void __launch_bounds__(NT, 1) pair_bwdc_kernel(TiledArgs a) {
    using M = Math<false>;
    constexpr int NW = NT / 32;
    constexpr int NV = 96;   // E, DE_1, DE_2: 16 complex each
    extern __shared__ __align__(16) unsigned char smem[];

    const DevPass* __restrict__ P = a.pass;
    const int w = P->w, ng = P->ng, ngates = P->n_gates, goff = P->gate_off;
    const int Lt = 1 << w;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s = blockIdx.y;
    const int mode = a.mode;
    const size_t A = (size_t)a.n_samples << a.n;
    const unsigned bytes = (unsigned)(Lt * 24);
    const unsigned wait_limit = a.copy_wait_limit ? a.copy_wait_limit : kPairWaitLimit;

    float4* sb4 = reinterpret_cast<float4*>(smem);
    float2* sb2 = reinterpret_cast<float2*>(sb4 + Lt);
    unsigned char* const buf0 = reinterpret_cast<unsigned char*>(sb2 + Lt);
    unsigned char* const buf1 = buf0 + bytes;
    float2* mats = reinterpret_cast<float2*>(buf1 + bytes);      // [gate][G^dag, V1^dag, V2^dag][16]
    float* wred = reinterpret_cast<float*>(mats + ngates * 48);
    float* acc = wred + 2 * NW * NV;                               // [ngates][NV]
    uint64_t* bars = reinterpret_cast<uint64_t*>(acc + ngates * NV);
    volatile int* stop = reinterpret_cast<volatile int*>(bars + 2);   // [step parity]
    int2* guv = reinterpret_cast<int2*>(bars + 3);

    stage_pair_mats(mats, a, goff, ngates, 2, 4);
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

    unsigned par = 0u, pend = 0u;
    const size_t sample_off = (size_t)s << a.n;
    TileCtx tc{0, P->off_lo, P->off_hi};

    for (int it = 0; it < a.tiles_per_cta; ++it) {
        const unsigned t = blockIdx.x * a.tiles_per_cta + it;
        tc.base = tile_base(P, t, sample_off, ng);
        if (tid == 0 && ngates > 0) {
            fence_proxy_async_smem();
            bulk_load_async(buf0, pair_cache_block(a, goff + ngates - 1, s, t, ng, Lt), bytes, &bars[0],
                            a.copy_extra_bytes);
            pend |= 1u;
            if (ngates > 1) {
                bulk_load_async(buf1, pair_cache_block(a, goff + ngates - 2, s, t, ng, Lt), bytes, &bars[1],
                                a.copy_extra_bytes);
                pend |= 2u;
            }
        }
        if (mode & M_LOAD_PHI) {   // co-states (phi, 0, 0); phi in the pass's output layout
            for (int m = tid; m < Lt; m += NT) {
                const size_t addr = tc.base + __ldg(&tc.offlo[m & 63]) + __ldg(&tc.offhi[m >> 6]);
                const unsigned l = swz(__ldg(&P->out_lo[m & 63]) | __ldg(&P->out_hi[m >> 6]));
                const float2 ph = a.phi[addr];
                sb4[l] = make_float4(ph.x, ph.y, 0.f, 0.f);
                sb2[l] = make_float2(0.f, 0.f);
            }
        } else {
            pair_load<NT>(sb4, sb2, a.cin, A, tc, P->out_lo, P->out_hi, Lt);
        }
        __syncthreads();   // the tile's co-states are in place before any warp starts a gate

        // One barrier per gate, as in the one-direction cached kernel: a thread
        // whose copy wait expires raises the stop flag of this step's parity and
        // goes on with the stale buffer; the flag is read after the barrier that
        // ends the step, which no later step's wait can precede.
        for (int i = 0; i < ngates; ++i) {
            const int g = ngates - 1 - i, b = i & 1;
            unsigned char* const cur = b ? buf1 : buf0;
            if (mbar_wait_bounded(&bars[b], (par >> b) & 1u, wait_limit)) {
                par ^= 1u << b;
                pend &= ~(1u << b);
            } else {
                stop[b] = 1;
                atomicOr(a.status, 2);
            }
            const float4* c4 = reinterpret_cast<const float4*>(cur);
            const float2* c2 = reinterpret_cast<const float2*>(c4 + Lt);
            const float2* Gh = mats + (g * 3) * 16;
            const float2* Vh1 = Gh + 16;
            const float2* Vh2 = Gh + 32;
            const int2 uv = guv[g];
            const int plo = min(uv.x, uv.y), phi_ = max(uv.x, uv.y);
            const unsigned mu = 1u << uv.x, mv = 1u << uv.y;
            float red[NV];
#pragma unroll
            for (int e = 0; e < NV; ++e) red[e] = 0.f;
            for (int q = tid; q < (Lt >> 2); q += NT) {
                const unsigned l0 = insert0(insert0(q, plo), phi_);
                const unsigned idx[4] = {swz(l0), swz(l0 | mv), swz(l0 | mu), swz(l0 | mu | mv)};
                float2 pp[4], d1[4], d2[4], Aa[4], B1[4], B2[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float4 x = c4[idx[c]];
                    const float4 y = sb4[idx[c]];
                    pp[c] = lo2(x); d1[c] = hi2(x); d2[c] = c2[idx[c]];
                    Aa[c] = lo2(y); B1[c] = hi2(y); B2[c] = sb2[idx[c]];
                }
#pragma unroll
                for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int e = 2 * (ii * 4 + j);
                        float2 v0 = make_float2(red[e], red[e + 1]);
                        M::cmac(v0, Aa[ii], pp[j], pp[j]);
                        red[e] = v0.x; red[e + 1] = v0.y;
                        float2 v1 = make_float2(red[32 + e], red[33 + e]);
                        M::cmac(v1, B1[ii], pp[j], pp[j]);
                        M::cmac(v1, Aa[ii], d1[j], d1[j]);
                        red[32 + e] = v1.x; red[33 + e] = v1.y;
                        float2 v2 = make_float2(red[64 + e], red[65 + e]);
                        M::cmac(v2, B2[ii], pp[j], pp[j]);
                        M::cmac(v2, Aa[ii], d2[j], d2[j]);
                        red[64 + e] = v2.x; red[65 + e] = v2.y;
                    }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    float2 na = make_float2(0.f, 0.f), n1 = na, n2 = na;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float2 gh = Gh[r * 4 + c];
                        M::mac(na, gh, Aa[c], Aa[c]);
                        M::mac(n1, gh, B1[c], B1[c]);
                        M::mac(n2, gh, B2[c], B2[c]);
                        M::mac(n1, Vh1[r * 4 + c], Aa[c], Aa[c]);
                        M::mac(n2, Vh2[r * 4 + c], Aa[c], Aa[c]);
                    }
                    sb4[idx[r]] = make_float4(na.x, na.y, n1.x, n1.y);
                    sb2[idx[r]] = n2;
                }
            }
            warp_reduce_scatter<NV>(red, lane);
            float* wr = wred + ((g & 1) * NW + warp) * NV;
#pragma unroll
            for (int k = 0; k < NV / 32; ++k) wr[lane * (NV / 32) + k] = red[k];
            __syncthreads();
            if (stop[b]) break;
            if (tid == 0 && i + 2 < ngates) {
                fence_proxy_async_smem();
                bulk_load_async(cur, pair_cache_block(a, goff + g - 2, s, t, ng, Lt), bytes, &bars[b],
                                a.copy_extra_bytes);
                pend |= 1u << b;
            }
            if (tid < NV) {
                float sum = 0.f;
#pragma unroll
                for (int ww = 0; ww < NW; ++ww) sum += wred[((g & 1) * NW + ww) * NV + tid];
                acc[g * NV + tid] += sum;
            }
        }
        if (stop[0] | stop[1]) break;
        if (mode & M_STORE_B) pair_store<NT>(a.cout, A, sb4, sb2, tc, P->in_lo, P->in_hi, Lt);
        __syncthreads();
    }

    if (stop[0] | stop[1]) {
        if (tid == 0)
            for (int j = 0; j < 2; ++j)
                if ((pend >> j) & 1u) mbar_wait_bounded(&bars[j], (par >> j) & 1u, wait_limit);
        return;
    }
    // (E, DE_1) to the first records, (E, DE_2) to the second.
    for (int i = tid; i < ngates * 64; i += NT) {
        const int g = i >> 6, e = i & 63;
        const int k = a.gates[goff + g].k;
        const size_t rec = (((size_t)k * a.n_samples + s) * a.cx_count + blockIdx.x) * 64;
        a.partial[rec + e] = (double)acc[g * NV + e];
        a.partial2[rec + e] = (double)acc[g * NV + (e < 32 ? e : e + 32)];
    }
}

}  // namespace

size_t pair_smem_bytes(bool bwd, int w, int threads, int max_gates) {
    const size_t Lt = (size_t)1 << w;
    if (!bwd) return Lt * 24 + (size_t)max_gates * 48 * 8;
    size_t b = 3 * Lt * 24;                                    // co-states + two cache buffers
    b += (size_t)max_gates * 48 * 8;                           // G^dag, V1^dag, V2^dag
    b += 2 * (size_t)(threads / 32) * 96 * 4;                  // cross-warp buffer
    b += (size_t)max_gates * 96 * 4;                           // FP32 sums
    b += 24 + (size_t)max_gates * 8;                           // mbarriers, stop flag, gate bits
    return b;
}

cudaError_t pair_set_smem_limits() {
    cudaError_t e = cudaFuncSetAttribute(pair_fwd_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(pair_bwdc_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

cudaError_t launch_pair(const TiledArgs& a, int w, int n_gates, cudaStream_t st) {
    const bool bwd = (a.mode & M_BWD) != 0;
    if ((a.mode & M_FWD) && bwd) return cudaErrorInvalidValue;
    const size_t smem = pair_smem_bytes(bwd, w, 256, n_gates);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    dim3 grid(a.cx_count, a.n_samples);
    if (bwd) pair_bwdc_kernel<256><<<grid, 256, smem, st>>>(a);
    else pair_fwd_kernel<256><<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace hvp
