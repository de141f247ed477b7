// Batched evaluation of many independent circuits of uneven size in one
// persistent launch.
//
// Work items are claimed in order from a global ticket. Circuits with n <= 12
// are "packed": one item holds 2^(12-n) samples in one 4096-amplitude tile
// (sample index = the address bits above the n qubit bits) and runs the whole
// circuit forward and back in shared memory. Larger circuits run window
// passes, one item per (pass, sample), each over all tiles of the sample;
// the items of one sample form a chain (phase f waits until phases 0..f-1 of
// that sample are done), and the ticket order (phase-major) guarantees that
// every awaited item was claimed earlier by a running CTA. Every wait is
// bounded; an expired wait sets an error flag and the host reports
// HVP_ETIMEOUT.
//
// Weighted co-states: the forward sweep ends with the overlaps T_s and
// Omega_s (Eq. overlap-general at the last cut, Eq. Omega as phi^dag dpsi^[K]),
// and the backward sweep starts from a = T_s phi_s, b = Omega_s phi_s. The
// environment sums of Eq. environment / Eq. Dpsi then come out already
// weighted, sum_a conj(a) psi = conj(T_s) E_s and
// sum_a conj(b) psi + conj(a) dpsi = conj(Omega_s) E_s + conj(T_s) DE_s, so
// they can be summed over samples inside an item:
//     grad C = -(2/N_s) conj(sum_s conj(T_s) E_s),
//     H C[V] = -(2/N_s) conj(sum_s conj(Omega_s) E_s + conj(T_s) DE_s).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hvp.h"
#include "tiled_common.cuh"

namespace hvp {

using namespace tile;

namespace {

constexpr int kBT = 256;          // threads of the batch kernel
constexpr int kBTile = 12;        // tile bits
constexpr int kBMaxPack = 1024;   // packed samples per tile at most (n >= 2)

struct BCircuit {
    int n, K, kofs, P, pass_ofs, packed, ns_real, ns_pad, sp, tiles, slots, done_ofs;
    size_t rec_ofs;                // records: [K][slots][64] doubles
    const float2* psi1q;           // ns_pad x n x 2
    const float2* phi;             // ns_pad x 2^n, layout of the last pass
    unsigned char* ckpt;           // boundaries 1..P (non-packed), each ns x 2^n x elt
    size_t ckpt_stride;            // bytes per boundary
    void* co;                      // co-states (non-packed)
    double2* T;                    // ns_pad
    double2* Om;                   // ns_pad
};

struct BItem { int c, f, s, dep; };

struct BatchArgs {
    const BCircuit* circ;
    const BItem* items;
    int n_items;
    const DevPass* passes;
    const DevGate* gates;
    const Mats32* mats;
    double* records;
    int* ticket;
    int* done;
    int* error;
    long long spin_limit;
    int dep_bias;       // added to every awaited count (0; 1 in the expired-wait test)
    int frob;           // Frobenius cost: co-state weights (1, 0) instead of (T_s, Omega_s)
};

// Block-wide sum of four FP32 values per thread into FP64 (red64 holds NW*4
// doubles of shared memory); every thread returns the totals.
__device__ __forceinline__ void block_sum4(float4 v, double* red64, double (&out)[4]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double d[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) d[i] += __shfl_xor_sync(0xffffffffu, d[i], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < 4; ++i) red64[warp * 4 + i] = d[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        double s = 0.0;
        for (int w = 0; w < kBT / 32; ++w) s += red64[w * 4 + i];
        out[i] = s;
    }
    __syncthreads();
}

// Flush FP32 per-gate sums of a pass into its FP64 record slot.
template <int NV>
__device__ __forceinline__ void flush_records(const BatchArgs& A, const BCircuit& C, const DevPass* P, float* acc,
                                              int slot) {
    const int ng = P->n_gates;
    for (int i = threadIdx.x; i < ng * 64; i += kBT) {
        const int g = i >> 6, e = i & 63;
        const int kl = A.gates[P->gate_off + g].k - C.kofs;
        A.records[C.rec_ofs + ((size_t)kl * C.slots + slot) * 64 + e] = e < NV ? (double)acc[g * NV + e] : 0.0;
    }
}

template <bool TAN>
__device__ __forceinline__ void stage_pass_mats(typename Math<false>::M* mats, const BatchArgs& A, const DevPass* P,
                                                int nmat) {
    const int which[6] = {1, 2, 5, 4, 0, 3};   // G^-1, G^dag, Y, V^dag, G, V
    TiledArgs ta{};
    ta.gates = A.gates;
    ta.mats = A.mats;
    stage_mats<false, kBT>(mats, ta, P->gate_off, P->n_gates, nmat, which);
}

template <bool TAN>
__device__ __forceinline__ void fwd_gates(typename Elt<TAN>::T* sf, const typename Math<false>::M* mats,
                                          const BatchArgs& A, const DevPass* P, int nmat, int Lt) {
    for (int g = 0; g < P->n_gates; ++g) {
        const DevGate dg = A.gates[P->gate_off + g];
        const auto* Gm = mats + (g * nmat + 4) * 16;
        const auto* Vm = mats + (g * nmat + 5) * 16;
        // 4096-amplitude tiles: four groups per thread, loop unrolled
        if (Lt == 4 * 4 * kBT) fwd_gate<TAN, false, kBT, const typename Math<false>::M*, 4>(sf, Gm, Vm, dg.u, dg.v, Lt);
        else fwd_gate<TAN, false, kBT>(sf, Gm, Vm, dg.u, dg.v, Lt);
        __syncthreads();
    }
}

template <bool TAN>
__device__ __forceinline__ void bwd_gates(typename Elt<TAN>::T* sf, typename Elt<TAN>::T* sb,
                                          const typename Math<false>::M* mats, float* wred, float* acc,
                                          const BatchArgs& A, const DevPass* P, int nmat, int Lt) {
    constexpr int NV = TAN ? 64 : 32;
    constexpr int NW = kBT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int g = P->n_gates - 1; g >= 0; --g) {
        const DevGate dg = A.gates[P->gate_off + g];
        const auto* base = mats + g * nmat * 16;
        float red[NV];
#pragma unroll
        for (int e = 0; e < NV; ++e) red[e] = 0.f;
        if (Lt == 4 * 4 * kBT)
            bwd_gate<TAN, false, kBT, NV, const typename Math<false>::M*, 4>(sf, sb, base, base + 16, base + 32,
                                                                            base + 48, dg.u, dg.v, Lt, red);
        else bwd_gate<TAN, false, kBT, NV>(sf, sb, base, base + 16, base + 32, base + 48, dg.u, dg.v, Lt, red);
        warp_reduce_scatter<NV>(red, lane);
        float* wr = wred + ((g & 1) * NW + warp) * 64;
#pragma unroll
        for (int i = 0; i < NV / 32; ++i) wr[lane * (NV / 32) + i] = red[i];
        __syncthreads();
        if (tid < NV) {
            float sum = 0.f;
#pragma unroll
            for (int w = 0; w < NW; ++w) sum += wred[((g & 1) * NW + w) * 64 + tid];
            acc[g * NV + tid] += sum;
        }
    }
    __syncthreads();
}

template <bool TAN>
__global__ void __launch_bounds__(kBT, 1) batch_kernel(BatchArgs A) {
    using E = typename Elt<TAN>::T;
    using MT = typename Math<false>::M;
    constexpr int NV = TAN ? 64 : 32;
    constexpr int NW = kBT / 32;
    constexpr int Lt = 1 << kBTile;
    extern __shared__ __align__(16) unsigned char smem[];
    E* sf = reinterpret_cast<E*>(smem);
    E* sb = sf + Lt;
    MT* mats = reinterpret_cast<MT*>(sb + Lt);
    float* wred = reinterpret_cast<float*>(mats + kMaxGatesPerPass * 6 * 16);
    float* acc = wred + 2 * NW * 64;
    double* red64 = reinterpret_cast<double*>(acc + kMaxGatesPerPass * NV);
    float2* tw = reinterpret_cast<float2*>(red64 + NW * 4);   // 2 x kBMaxPack
    __shared__ int s_item, s_abort;
    const int tid = threadIdx.x;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(A.ticket, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= A.n_items) break;
        const BItem I = A.items[it];
        const BCircuit C = A.circ[I.c];
        if (tid == 0) {
            s_abort = 0;
            if (I.dep > 0) {
                volatile int* d = A.done + C.done_ofs + I.s;
                long long spins = 0;
                volatile int* errflag = A.error;
                while (*d < I.dep + A.dep_bias) {
                    __nanosleep(200);
                    // bounded wait: report and move on; after the first expired
                    // wait every later wait gives up at once
                    if (++spins > A.spin_limit || *errflag) {
                        atomicOr(A.error, 2);
                        s_abort = 1;
                        break;
                    }
                }
                __threadfence();
            }
        }
        __syncthreads();
        if (!s_abort) {
            const size_t dim = (size_t)1 << C.n;
            if (C.packed) {
                // ---------------- whole circuit for sp samples in one tile
                const int j = I.s;                               // item index
                const size_t base = (size_t)j * C.sp * dim;      // contiguous samples
                const DevPass* P0 = A.passes + C.pass_ofs;
                TileCtx tc{base, P0->off_lo, P0->off_hi};
                gen_tile<E, kBT>(sf, P0, C.psi1q + (size_t)j * C.sp * C.n * 2, 0, C.n, 0, Lt, C.n);
                __syncthreads();
                for (int p = 0; p < C.P; ++p) {
                    const DevPass* P = A.passes + C.pass_ofs + p;
                    stage_pass_mats<TAN>(mats, A, P, 6);
                    __syncthreads();
                    fwd_gates<TAN>(sf, mats, A, P, 6, Lt);
                }
                // reference states into the co-state tile
                for (int m = tid; m < Lt; m += kBT) {
                    const unsigned l = __ldg(&P0->in_lo[m & 63]) | __ldg(&P0->in_hi[m >> 6]);
                    const float2 ph = __ldcg(C.phi + base + __ldg(&P0->off_lo[m & 63]) + __ldg(&P0->off_hi[m >> 6]));
                    if constexpr (TAN) sb[swz(l)] = make_float4(ph.x, ph.y, 0.f, 0.f);
                    else sb[swz(l)] = ph;
                }
                __syncthreads();
                // overlaps per packed sample: T = phi^dag psi, Omega = phi^dag dpsi
                for (int q = 0; q < C.sp; ++q) {
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    for (int t = tid; t < (int)dim; t += kBT) {
                        const unsigned l = swz(((unsigned)q << C.n) + t);
                        float2 ph, ps, dps = make_float2(0.f, 0.f);
                        if constexpr (TAN) { ph = lo2(sb[l]); ps = lo2(sf[l]); dps = hi2(sf[l]); }
                        else { ph = sb[l]; ps = sf[l]; }
                        v.x += ph.x * ps.x + ph.y * ps.y;  v.y += ph.x * ps.y - ph.y * ps.x;
                        v.z += ph.x * dps.x + ph.y * dps.y; v.w += ph.x * dps.y - ph.y * dps.x;
                    }
                    double tot[4];
                    block_sum4(v, red64, tot);
                    if (tid == 0) {
                        const int s = j * C.sp + q;
                        C.T[s] = make_double2(tot[0], tot[1]);
                        C.Om[s] = make_double2(tot[2], tot[3]);
                        tw[2 * q] = A.frob ? make_float2(1.f, 0.f) : make_float2((float)tot[0], (float)tot[1]);
                        tw[2 * q + 1] = A.frob ? make_float2(0.f, 0.f) : make_float2((float)tot[2], (float)tot[3]);
                    }
                }
                __syncthreads();
                // weighted co-states a = T phi, b = Omega phi
                for (int l = tid; l < Lt; l += kBT) {
                    const int q = l >> C.n;
                    const float2 Tq = tw[2 * q], Oq = tw[2 * q + 1];
                    const unsigned sl = swz(l);
                    if constexpr (TAN) {
                        const float2 ph = lo2(sb[sl]);
                        sb[sl] = make_float4(Tq.x * ph.x - Tq.y * ph.y, Tq.x * ph.y + Tq.y * ph.x,
                                             Oq.x * ph.x - Oq.y * ph.y, Oq.x * ph.y + Oq.y * ph.x);
                    } else {
                        const float2 ph = sb[sl];
                        sb[sl] = make_float2(Tq.x * ph.x - Tq.y * ph.y, Tq.x * ph.y + Tq.y * ph.x);
                    }
                }
                __syncthreads();
                for (int p = C.P - 1; p >= 0; --p) {
                    const DevPass* P = A.passes + C.pass_ofs + p;
                    stage_pass_mats<TAN>(mats, A, P, 6);
                    for (int i = tid; i < P->n_gates * NV; i += kBT) acc[i] = 0.f;
                    __syncthreads();
                    bwd_gates<TAN>(sf, sb, mats, wred, acc, A, P, 6, Lt);
                    flush_records<NV>(A, C, P, acc, j);
                    __syncthreads();
                }
            } else if (I.f < C.P) {
                // ---------------- forward pass p of one sample, all tiles
                const int p = I.f, s = I.s;
                const DevPass* P = A.passes + C.pass_ofs + p;
                const int Lp = 1 << P->w;
                const E* xin = p == 0 ? nullptr : reinterpret_cast<const E*>(C.ckpt + (size_t)(p - 1) * C.ckpt_stride);
                E* xout = reinterpret_cast<E*>(C.ckpt + (size_t)p * C.ckpt_stride);
                stage_pass_mats<TAN>(mats, A, P, 6);
                __syncthreads();
                double tot_acc[4] = {0.0, 0.0, 0.0, 0.0};
                for (int t = 0; t < C.tiles; ++t) {
                    const size_t base = tile_base(P, t, (size_t)s << C.n, P->ng);
                    TileCtx tc{base, P->off_lo, P->off_hi};
                    if (p == 0) gen_tile<E, kBT>(sf, P, C.psi1q + (size_t)s * C.n * 2, t, P->nq, P->ng, Lp, C.n);
                    else load_tile<E, kBT, true>(sf, xin, tc, P->in_lo, P->in_hi, Lp);
                    __syncthreads();
                    fwd_gates<TAN>(sf, mats, A, P, 6, Lp);
                    store_tile<E, kBT>(xout, sf, tc, P->out_lo, P->out_hi, Lp);
                    if (p == C.P - 1) {   // overlaps at the last cut
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        for (int m = tid; m < Lp; m += kBT) {
                            const unsigned l = __ldg(&P->out_lo[m & 63]) | __ldg(&P->out_hi[m >> 6]);
                            const float2 ph = __ldcg(C.phi + base + __ldg(&P->off_lo[m & 63]) + __ldg(&P->off_hi[m >> 6]));
                            float2 ps, dps = make_float2(0.f, 0.f);
                            if constexpr (TAN) { ps = lo2(sf[swz(l)]); dps = hi2(sf[swz(l)]); }
                            else ps = sf[swz(l)];
                            v.x += ph.x * ps.x + ph.y * ps.y;  v.y += ph.x * ps.y - ph.y * ps.x;
                            v.z += ph.x * dps.x + ph.y * dps.y; v.w += ph.x * dps.y - ph.y * dps.x;
                        }
                        double tot[4];
                        block_sum4(v, red64, tot);
                        for (int i = 0; i < 4; ++i) tot_acc[i] += tot[i];
                    }
                    __syncthreads();
                }
                if (p == C.P - 1 && tid == 0) {
                    C.T[s] = make_double2(tot_acc[0], tot_acc[1]);
                    C.Om[s] = make_double2(tot_acc[2], tot_acc[3]);
                }
            } else {
                // ---------------- backward pass p of one sample, all tiles
                const int p = 2 * C.P - 1 - I.f, s = I.s;
                const DevPass* P = A.passes + C.pass_ofs + p;
                const int Lp = 1 << P->w;
                const E* xin = reinterpret_cast<const E*>(C.ckpt + (size_t)p * C.ckpt_stride);
                E* co = reinterpret_cast<E*>(C.co);
                const double2 Ts = __ldcg(C.T + s), Os = __ldcg(C.Om + s);
                const float2 Tq = A.frob ? make_float2(1.f, 0.f) : make_float2((float)Ts.x, (float)Ts.y);
                const float2 Oq = A.frob ? make_float2(0.f, 0.f) : make_float2((float)Os.x, (float)Os.y);
                stage_pass_mats<TAN>(mats, A, P, 4);
                for (int i = tid; i < P->n_gates * NV; i += kBT) acc[i] = 0.f;
                __syncthreads();
                for (int t = 0; t < C.tiles; ++t) {
                    const size_t base = tile_base(P, t, (size_t)s << C.n, P->ng);
                    TileCtx tc{base, P->off_lo, P->off_hi};
                    load_tile<E, kBT, true>(sf, xin, tc, P->out_lo, P->out_hi, Lp);
                    if (p == C.P - 1) {
                        for (int m = tid; m < Lp; m += kBT) {
                            const unsigned l = __ldg(&P->out_lo[m & 63]) | __ldg(&P->out_hi[m >> 6]);
                            const float2 ph = __ldcg(C.phi + base + __ldg(&P->off_lo[m & 63]) + __ldg(&P->off_hi[m >> 6]));
                            const float2 a = make_float2(Tq.x * ph.x - Tq.y * ph.y, Tq.x * ph.y + Tq.y * ph.x);
                            if constexpr (TAN)
                                sb[swz(l)] = make_float4(a.x, a.y, Oq.x * ph.x - Oq.y * ph.y, Oq.x * ph.y + Oq.y * ph.x);
                            else sb[swz(l)] = a;
                        }
                    } else {
                        load_tile<E, kBT, true>(sb, co, tc, P->out_lo, P->out_hi, Lp);
                    }
                    __syncthreads();
                    bwd_gates<TAN>(sf, sb, mats, wred, acc, A, P, 4, Lp);
                    if (p > 0) store_tile<E, kBT>(co, sb, tc, P->in_lo, P->in_hi, Lp);
                    __syncthreads();
                }
                flush_records<NV>(A, C, P, acc, s);
            }
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            if (!C.packed) atomicAdd(A.done + C.done_ofs + I.s, 1);
        }
    }
}

// grad / HVP per gate from the weighted records, then App. F; block = gate.
__device__ __forceinline__ double2 dmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 dconj(double2 a) { return make_double2(a.x, -a.y); }

__global__ void bpost_grad_kernel(const BCircuit* __restrict__ circ, const int* __restrict__ gate_circ,
                                  const double* __restrict__ records, const double2* __restrict__ G,
                                  const double2* __restrict__ V, double2* ge, double2* he, double2* gr, double2* hr,
                                  int tangent, int frob) {
    const int k = blockIdx.x, e = threadIdx.x;
    const BCircuit& C = circ[gate_circ[k]];
    const int kl = k - C.kofs;
    __shared__ double2 sG[16], sV[16], sg[16], sX[16];
    double2 RE = make_double2(0.0, 0.0), RD = make_double2(0.0, 0.0);
    const double* rec = records + C.rec_ofs + (size_t)kl * C.slots * 64;
    for (int s = 0; s < C.slots; ++s) {
        RE.x += rec[(size_t)s * 64 + 2 * e];
        RE.y += rec[(size_t)s * 64 + 2 * e + 1];
        RD.x += rec[(size_t)s * 64 + 32 + 2 * e];
        RD.y += rec[(size_t)s * 64 + 32 + 2 * e + 1];
    }
    const double scale = (frob ? -1.0 : -2.0) / C.ns_real;
    const double2 g = make_double2(scale * RE.x, -scale * RE.y);   // -(2/N) conj(sum conj(T) E)
    const double2 h = make_double2(scale * RD.x, -scale * RD.y);
    sG[e] = G[k * 16 + e];
    sV[e] = tangent ? V[k * 16 + e] : make_double2(0.0, 0.0);
    sg[e] = g;
    ge[k * 16 + e] = g;
    if (tangent) he[k * 16 + e] = h;
    __syncthreads();
    const int r = e >> 2, c = e & 3;
    auto abdc = [&](const double2* Am, const double2* Bm, const double2* Cm) {
        double2 a = make_double2(0.0, 0.0);
        for (int x = 0; x < 4; ++x)
            for (int y = 0; y < 4; ++y) {
                const double2 t = dmul(dmul(Am[r * 4 + x], dconj(Bm[y * 4 + x])), Cm[y * 4 + c]);
                a.x += t.x;
                a.y += t.y;
            }
        return a;
    };
    const double2 gg = abdc(sG, sg, sG);
    gr[k * 16 + e] = make_double2(0.5 * g.x - 0.5 * gg.x, 0.5 * g.y - 0.5 * gg.y);
    if (tangent) {
        const double2 t1 = abdc(sV, sg, sG), t2 = abdc(sG, sg, sV);
        const double2 x = make_double2(h.x - 0.5 * t1.x - 0.5 * t2.x, h.y - 0.5 * t1.y - 0.5 * t2.y);
        sX[e] = x;
        __syncthreads();
        const double2 xx = abdc(sG, sX, sG);
        hr[k * 16 + e] = make_double2(0.5 * x.x - 0.5 * xx.x, 0.5 * x.y - 0.5 * xx.y);
    }
}

__global__ void bpost_loss_kernel(const BCircuit* __restrict__ circ, double* loss, int frob) {
    const BCircuit& C = circ[blockIdx.x];
    __shared__ double sh[256];
    double a = 0.0;
    for (int s = threadIdx.x; s < C.ns_real; s += blockDim.x)
        a += frob ? C.T[s].x : C.T[s].x * C.T[s].x + C.T[s].y * C.T[s].y;
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss[blockIdx.x] = 1.0 - sh[0] / C.ns_real;   // Eq. costHS
}

size_t batch_smem(bool tan) {
    const size_t elt = tan ? 16 : 8;
    const int NV = tan ? 64 : 32;
    return 2 * (elt << kBTile) + (size_t)kMaxGatesPerPass * 6 * 16 * 8 + 2 * (kBT / 32) * 64 * 4 +
           (size_t)kMaxGatesPerPass * NV * 4 + (kBT / 32) * 4 * 8 + 2 * kBMaxPack * 8;
}

}  // namespace

// ------------------------------------------------------------------ host side

struct BatchImpl {
    int nc = 0, sumK = 0, sumNs = 0, n_items = 0, grid = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    int flags = 0;
    int window = kBTile;        // window qubits of the circuits above kBTile qubits
    long long spin_limit = 20000000;   // x 200 ns sleeps: a few seconds at most
    int dep_bias = 0;
    std::vector<BCircuit> circ;
    std::vector<int> K, kofs, ns;
    std::vector<void*> allocs;
    size_t bytes = 0;
    BCircuit* d_circ = nullptr;
    BItem* d_items = nullptr;
    DevPass* d_passes = nullptr;
    DevGate* d_gates = nullptr;
    Mats32* d_mats = nullptr;
    double2* d_G = nullptr;
    double2* d_V = nullptr;
    int* d_gate_circ = nullptr;
    double* d_records = nullptr;
    int* d_sync = nullptr;      // [ticket, error, done...]
    int sync_len = 0;
    int* d_status = nullptr;
    double* d_res = nullptr;    // loss[nc] | ge | he | gr | hr
    double* h_in = nullptr;
    double* h_res = nullptr;
    int* h_flags = nullptr;     // [status, error]
    size_t res_len = 0;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int launches = 0;

    // the per-gate blocks are double2 arrays: start them on a 16-byte boundary
    // after the nc losses (an odd nc would misalign them)
    size_t off_ge() const { return ((size_t)nc + 1) & ~(size_t)1; }
    size_t off_he() const { return off_ge() + 32 * (size_t)sumK; }
    size_t off_gr() const { return off_he() + 32 * (size_t)sumK; }
    size_t off_hr() const { return off_gr() + 32 * (size_t)sumK; }
};

namespace {

#define B_TRY(call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);                      \
            return e_ == cudaErrorMemoryAllocation ? HVP_ENOMEM : HVP_ECUDA;               \
        }                                                                                  \
    } while (0)

int balloc(BatchImpl* b, void** p, size_t bytes, std::string& err) {
    *p = nullptr;
    if (!bytes) return HVP_OK;
    if (b->bytes + bytes > device_alloc_cap()) {
        err = "device allocation of " + std::to_string(bytes) + " bytes exceeds the cap HVP_DEVICE_ALLOC_CAP_MB";
        return HVP_ENOMEM;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        err = "cudaMalloc of " + std::to_string(bytes) + " bytes failed";
        return HVP_ENOMEM;
    }
    b->allocs.push_back(*p);
    b->bytes += bytes;
    return HVP_OK;
}

// Pass descriptor of a packed tile: the n qubit bits in the standard layout
// (qubit q on address bit n-1-q) and 12-n sample bits above them.
DevPass packed_pass(const Plan& plan, const PassPlan& pp, int gate_off, int n_gates) {
    DevPass d{};
    const int n = plan.n;
    d.w = kBTile;
    d.nq = n;
    d.ng = 0;
    d.n_gates = n_gates;
    d.gate_off = gate_off;
    for (int j = 0; j < n; ++j) d.sq[j] = pp.S[j];
    auto jbit = [&](int q) { return (int)(std::find(pp.S.begin(), pp.S.end(), q) - pp.S.begin()); };
    auto smem_bit_of_rank = [&](int t) { return t < n ? jbit(n - 1 - t) : t; };   // rank t = address bit t
    for (int x = 0; x < 64; ++x) {
        uint32_t off = 0, li = 0;
        for (int t = 0; t < 6; ++t)
            if ((x >> t) & 1) { off |= 1u << t; li |= 1u << smem_bit_of_rank(t); }
        d.off_lo[x] = off; d.in_lo[x] = (uint16_t)li; d.out_lo[x] = (uint16_t)li;
    }
    for (int y = 0; y < 256; ++y) {
        uint32_t off = 0, li = 0;
        for (int t = 6; t < kBTile; ++t)
            if ((y >> (t - 6)) & 1) { off |= 1u << t; li |= 1u << smem_bit_of_rank(t); }
        d.off_hi[y] = off; d.in_hi[y] = (uint16_t)li; d.out_hi[y] = (uint16_t)li;
    }
    return d;
}

int enqueue_batch(BatchImpl* b, bool tan, std::string& err) {
    cudaStream_t st = b->stream;
    B_TRY(cudaMemsetAsync(b->d_sync, 0, sizeof(int) * b->sync_len, st));
    B_TRY(cudaMemsetAsync(b->d_status, 0, sizeof(int), st));
    B_TRY(launch_prep(b->d_G, tan ? b->d_V : nullptr, b->d_mats, false, b->sumK, b->d_status, st));
    BatchArgs A{};
    A.circ = b->d_circ;
    A.items = b->d_items;
    A.n_items = b->n_items;
    A.passes = b->d_passes;
    A.gates = b->d_gates;
    A.mats = b->d_mats;
    A.records = b->d_records;
    A.ticket = b->d_sync;
    A.error = b->d_sync + 1;
    A.done = b->d_sync + 2;
    A.spin_limit = b->spin_limit;
    A.dep_bias = b->dep_bias;
    A.frob = (b->flags & HVP_FROBENIUS) ? 1 : 0;
    const size_t smem = batch_smem(tan);
    if (tan) batch_kernel<true><<<b->grid, kBT, smem, st>>>(A);
    else batch_kernel<false><<<b->grid, kBT, smem, st>>>(A);
    B_TRY(cudaGetLastError());
    bpost_grad_kernel<<<b->sumK, 16, 0, st>>>(b->d_circ, b->d_gate_circ, b->d_records, b->d_G, b->d_V,
                                              reinterpret_cast<double2*>(b->d_res + b->off_ge()),
                                              reinterpret_cast<double2*>(b->d_res + b->off_he()),
                                              reinterpret_cast<double2*>(b->d_res + b->off_gr()),
                                              reinterpret_cast<double2*>(b->d_res + b->off_hr()), tan ? 1 : 0,
                                              A.frob);
    bpost_loss_kernel<<<b->nc, 256, 0, st>>>(b->d_circ, b->d_res, A.frob);
    B_TRY(cudaGetLastError());
    b->launches = 4;
    return HVP_OK;
}

int run_batch(BatchImpl* b, bool tan, bool graphs, std::string& err) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    B_TRY(cudaStreamIsCapturing(b->stream, &cap));
    if (!graphs || cap != cudaStreamCaptureStatusNone) return enqueue_batch(b, tan, err);
    cudaGraphExec_t& ge = b->gexec[tan ? 1 : 0];
    if (!ge) {
        cudaGraph_t g = nullptr;
        B_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_batch(b, tan, err);
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        B_TRY(e);
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { ge = nullptr; B_TRY(e); }
    }
    B_TRY(cudaGraphLaunch(ge, b->stream));
    return HVP_OK;
}

}  // namespace

int batch_init(BatchImpl** out, int nc, const hvp_config* cfgs, const double* const* psi_1q,
               const double* const* ref, cudaStream_t stream, int window, std::string& err) {
    *out = nullptr;
    BatchImpl* b = new BatchImpl();
    auto bail = [&](int rc) { batch_free(b); return rc; };
#undef B_TRY
#define B_TRY(call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);                      \
            return bail(e_ == cudaErrorMemoryAllocation ? HVP_ENOMEM : HVP_ECUDA);         \
        }                                                                                  \
    } while (0)
    b->nc = nc;
    b->stream = stream;
    b->device = cfgs[0].device;
    b->flags = cfgs[0].flags;
    b->window = window > 0 ? std::min(window, kBTile) : kBTile;
    if (b->window < 6) { err = "batch: window below 6 qubits"; return bail(HVP_EINVAL); }
    std::vector<Plan> plans(nc);
    std::vector<DevPass> passes;
    std::vector<DevGate> gates;
    std::vector<int> gate_circ;
    b->circ.resize(nc);
    int sumK = 0, done_total = 0;
    for (int c = 0; c < nc; ++c) {
        const hvp_config& cf = cfgs[c];
        BCircuit& C = b->circ[c];
        C = BCircuit{};
        C.n = cf.n;
        C.K = num_gates(cf.n, cf.n_layers);
        C.kofs = sumK;
        sumK += C.K;
        C.ns_real = cf.n_samples;
        C.packed = cf.n <= kBTile;
        // packed circuits hold all their qubits in one tile; larger ones run
        // window passes of b->window qubits
        const int wc = C.packed ? cf.n : std::min(cf.n, b->window);
        int rc = make_plan(cf.n, cf.n_layers, wc, std::min(kLowBits, wc - 1), plans[c]);
        if (rc) { err = "batch: planning failed for circuit " + std::to_string(c); return bail(rc); }
        const Plan& pl = plans[c];
        C.P = (int)pl.passes.size();
        if (!C.packed && C.P > 30) { err = "batch: too many passes"; return bail(HVP_EINVAL); }
        C.pass_ofs = (int)passes.size();
        if (C.packed) {
            C.sp = 1 << (kBTile - cf.n);
            C.ns_pad = (cf.n_samples + C.sp - 1) / C.sp * C.sp;
            C.tiles = 1;
            C.slots = C.ns_pad / C.sp;
            for (auto& pp : pl.passes) {
                passes.push_back(packed_pass(pl, pp, (int)gates.size(), (int)pp.gates.size()));
                for (int g : pp.gates) {
                    DevGate dg{};
                    dg.k = C.kofs + g;
                    dg.u = (int)(std::find(pp.S.begin(), pp.S.end(), pl.first_qubit[g]) - pp.S.begin());
                    dg.v = (int)(std::find(pp.S.begin(), pp.S.end(), pl.first_qubit[g] + 1) - pp.S.begin());
                    gates.push_back(dg);
                }
            }
        } else {
            C.sp = 1;
            C.ns_pad = cf.n_samples;
            C.tiles = 1 << (cf.n - wc);
            C.slots = cf.n_samples;
            std::vector<DevPass> dp;
            std::vector<DevGate> dg;
            build_dev_passes(pl, dp, dg);
            const int goff = (int)gates.size();
            for (auto& d : dp) { d.gate_off += goff; passes.push_back(d); }
            for (auto& g : dg) { g.k += C.kofs; gates.push_back(g); }
            C.done_ofs = done_total;
            done_total += cf.n_samples;
        }
        for (int k = 0; k < C.K; ++k) gate_circ.push_back(c);
        b->K.push_back(C.K);
        b->kofs.push_back(C.kofs);
        b->ns.push_back(C.ns_real);
    }
    b->sumK = sumK;
    for (int x : b->ns) b->sumNs += x;

    // Device buffers.
    int rc;
    size_t rec_total = 0;
    for (auto& C : b->circ) { C.rec_ofs = rec_total; rec_total += (size_t)C.K * C.slots * 64; }
    if ((rc = balloc(b, (void**)&b->d_records, sizeof(double) * rec_total, err))) return bail(rc);
    if ((rc = balloc(b, (void**)&b->d_G, 256 * (size_t)sumK, err))) return bail(rc);
    if ((rc = balloc(b, (void**)&b->d_V, 256 * (size_t)sumK, err))) return bail(rc);
    if ((rc = balloc(b, (void**)&b->d_mats, sizeof(Mats32) * (size_t)sumK, err))) return bail(rc);
    if ((rc = balloc(b, (void**)&b->d_passes, sizeof(DevPass) * passes.size(), err))) return bail(rc);
    if ((rc = balloc(b, (void**)&b->d_gates, sizeof(DevGate) * gates.size(), err))) return bail(rc);
    if ((rc = balloc(b, (void**)&b->d_gate_circ, sizeof(int) * gate_circ.size(), err))) return bail(rc);
    b->sync_len = 2 + std::max(done_total, 1);
    if ((rc = balloc(b, (void**)&b->d_sync, sizeof(int) * b->sync_len, err))) return bail(rc);
    if ((rc = balloc(b, (void**)&b->d_status, sizeof(int), err))) return bail(rc);
    b->res_len = b->off_hr() + 32 * (size_t)sumK;
    if ((rc = balloc(b, (void**)&b->d_res, sizeof(double) * b->res_len, err))) return bail(rc);
    B_TRY(cudaMemset(b->d_V, 0, 256 * (size_t)sumK));
    B_TRY(cudaMallocHost((void**)&b->h_in, sizeof(double) * 64 * (size_t)sumK));
    B_TRY(cudaMallocHost((void**)&b->h_res, sizeof(double) * b->res_len));
    B_TRY(cudaMallocHost((void**)&b->h_flags, sizeof(int) * 2));
    B_TRY(cudaMemcpy(b->d_passes, passes.data(), sizeof(DevPass) * passes.size(), cudaMemcpyHostToDevice));
    B_TRY(cudaMemcpy(b->d_gates, gates.data(), sizeof(DevGate) * gates.size(), cudaMemcpyHostToDevice));
    B_TRY(cudaMemcpy(b->d_gate_circ, gate_circ.data(), sizeof(int) * gate_circ.size(), cudaMemcpyHostToDevice));

    std::vector<BItem> items;
    for (int c = 0; c < nc; ++c) {
        BCircuit& C = b->circ[c];
        const size_t dim = (size_t)1 << C.n;
        // inputs: psi_1q (zero-padded samples give zero states) and phi
        std::vector<float2> q((size_t)C.ns_pad * C.n * 2, make_float2(0.f, 0.f));
        for (size_t i = 0; i < (size_t)C.ns_real * C.n * 2; ++i)
            q[i] = make_float2((float)psi_1q[c][2 * i], (float)psi_1q[c][2 * i + 1]);
        void* p = nullptr;
        if ((rc = balloc(b, &p, sizeof(float2) * q.size(), err))) return bail(rc);
        C.psi1q = (const float2*)p;
        B_TRY(cudaMemcpy(p, q.data(), sizeof(float2) * q.size(), cudaMemcpyHostToDevice));
        if ((rc = balloc(b, &p, sizeof(float2) * dim * C.ns_pad, err))) return bail(rc);
        C.phi = (const float2*)p;
        B_TRY(cudaMemset(p, 0, sizeof(float2) * dim * C.ns_pad));
        {
            // phi_s = U_ref psi_s with a single-circuit context (same plan and layout),
            // or the given reference states permuted into the last pass's layout.
            hvp_config sc = cfgs[c];
            sc.flags = (cfgs[c].flags & HVP_PHI_GIVEN) | HVP_NO_GRAPH;
            sc.precision = HVP_C64;
            sc.window = C.packed ? 0 : b->window;   // the plan used here
            sc.threads = 256;
            sc.variant = 1;
            sc.checkpoint_stride = 0;
            sc.stream = stream;
            hvp_ctx* tmp = nullptr;
            int r2 = hvp_init(&tmp, &sc, psi_1q[c], ref[c]);
            if (r2) { err = std::string("batch: reference states of circuit ") + std::to_string(c) + ": " + hvp_last_error(nullptr); return bail(r2); }
            r2 = hvp_internal_copy_phi(tmp, p, sizeof(float2) * dim * C.ns_real);
            hvp_free(tmp);
            if (r2) { err = "batch: copying reference states failed"; return bail(r2); }
        }
        if ((rc = balloc(b, &p, sizeof(double2) * C.ns_pad, err))) return bail(rc);
        C.T = (double2*)p;
        B_TRY(cudaMemset(p, 0, sizeof(double2) * C.ns_pad));
        if ((rc = balloc(b, &p, sizeof(double2) * C.ns_pad, err))) return bail(rc);
        C.Om = (double2*)p;
        B_TRY(cudaMemset(p, 0, sizeof(double2) * C.ns_pad));
        if (C.packed) {
            for (int j = 0; j < C.slots; ++j) items.push_back(BItem{c, 0, j, 0});
        } else {
            C.ckpt_stride = 16 * dim * C.ns_real;
            if ((rc = balloc(b, &p, C.ckpt_stride * C.P, err))) return bail(rc);
            C.ckpt = (unsigned char*)p;
            if ((rc = balloc(b, &C.co, 16 * dim * C.ns_real, err))) return bail(rc);
            for (int f = 0; f < 2 * C.P; ++f)
                for (int s = 0; s < C.ns_real; ++s) items.push_back(BItem{c, f, s, f});
        }
    }
    // Phase-major ticket order: every awaited item has a smaller ticket.
    std::stable_sort(items.begin(), items.end(), [](const BItem& x, const BItem& y) { return x.f < y.f; });
    b->n_items = (int)items.size();
    if ((rc = balloc(b, (void**)&b->d_items, sizeof(BItem) * items.size(), err))) return bail(rc);
    B_TRY(cudaMemcpy(b->d_items, items.data(), sizeof(BItem) * items.size(), cudaMemcpyHostToDevice));
    if ((rc = balloc(b, (void**)&b->d_circ, sizeof(BCircuit) * nc, err))) return bail(rc);
    B_TRY(cudaMemcpy(b->d_circ, b->circ.data(), sizeof(BCircuit) * nc, cudaMemcpyHostToDevice));

    B_TRY(cudaFuncSetAttribute(batch_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem(true)));
    B_TRY(cudaFuncSetAttribute(batch_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem(false)));
    int per_sm = 0, sms = 0;
    B_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<true>, kBT, batch_smem(true)));
    B_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    b->grid = std::max(1, per_sm) * sms;
    B_TRY(cudaDeviceSynchronize());
    *out = b;
    return HVP_OK;
}
#undef B_TRY
#define B_TRY(call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);                      \
            return e_ == cudaErrorMemoryAllocation ? HVP_ENOMEM : HVP_ECUDA;               \
        }                                                                                  \
    } while (0)

int batch_call(BatchImpl* b, const double* G, const double* V, bool dev, double* loss, double* grad, double* hvp,
               std::string& err) {
    const size_t n32 = 32 * (size_t)b->sumK;
    const bool tan = V != nullptr;
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (!dev) {
        std::memcpy(b->h_in, G, sizeof(double) * n32);
        if (tan) std::memcpy(b->h_in + n32, V, sizeof(double) * n32);
    }
    B_TRY(cudaMemcpyAsync(b->d_G, dev ? G : b->h_in, sizeof(double) * n32, kind, b->stream));
    if (tan) B_TRY(cudaMemcpyAsync(b->d_V, dev ? V : b->h_in + n32, sizeof(double) * n32, kind, b->stream));
    int rc = run_batch(b, tan, !(b->flags & HVP_NO_GRAPH), err);
    if (rc) return rc;
    const bool riem = (b->flags & HVP_RIEMANNIAN) != 0;
    const double* dg = b->d_res + (riem ? b->off_gr() : b->off_ge());
    const double* dh = b->d_res + (riem ? b->off_hr() : b->off_he());
    if (dev) {
        if (loss) B_TRY(cudaMemcpyAsync(loss, b->d_res, sizeof(double) * b->nc, cudaMemcpyDeviceToDevice, b->stream));
        if (grad) B_TRY(cudaMemcpyAsync(grad, dg, sizeof(double) * n32, cudaMemcpyDeviceToDevice, b->stream));
        if (hvp && tan) B_TRY(cudaMemcpyAsync(hvp, dh, sizeof(double) * n32, cudaMemcpyDeviceToDevice, b->stream));
        return HVP_OK;
    }
    B_TRY(cudaMemcpyAsync(b->h_res, b->d_res, sizeof(double) * b->res_len, cudaMemcpyDeviceToHost, b->stream));
    B_TRY(cudaMemcpyAsync(b->h_flags, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    B_TRY(cudaMemcpyAsync(b->h_flags + 1, b->d_sync + 1, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    B_TRY(cudaStreamSynchronize(b->stream));
    if (b->h_flags[1]) { err = "batch: a bounded device-side wait expired"; return HVP_ETIMEOUT; }
    if (b->h_flags[0]) { err = "batch: a gate is singular or not finite"; return HVP_ENONFINITE; }
    const double* hg = b->h_res + (riem ? b->off_gr() : b->off_ge());
    const double* hh = b->h_res + (riem ? b->off_hr() : b->off_he());
    for (size_t i = 0; i < (size_t)b->nc; ++i)
        if (!std::isfinite(b->h_res[i])) { err = "batch: non-finite result"; return HVP_ENONFINITE; }
    if (loss) std::memcpy(loss, b->h_res, sizeof(double) * b->nc);
    if (grad) std::memcpy(grad, hg, sizeof(double) * n32);
    if (hvp && tan) std::memcpy(hvp, hh, sizeof(double) * n32);
    return HVP_OK;
}

int batch_get(BatchImpl* b, int what, double* out, std::string& err) {
    const size_t n32 = 32 * (size_t)b->sumK;
    B_TRY(cudaStreamSynchronize(b->stream));
    switch (what) {
        case HVP_OUT_LOSS: B_TRY(cudaMemcpy(out, b->d_res, sizeof(double) * b->nc, cudaMemcpyDeviceToHost)); return HVP_OK;
        case HVP_OUT_GRAD_E: B_TRY(cudaMemcpy(out, b->d_res + b->off_ge(), sizeof(double) * n32, cudaMemcpyDeviceToHost)); return HVP_OK;
        case HVP_OUT_HVP_E: B_TRY(cudaMemcpy(out, b->d_res + b->off_he(), sizeof(double) * n32, cudaMemcpyDeviceToHost)); return HVP_OK;
        case HVP_OUT_GRAD_R: B_TRY(cudaMemcpy(out, b->d_res + b->off_gr(), sizeof(double) * n32, cudaMemcpyDeviceToHost)); return HVP_OK;
        case HVP_OUT_HVP_R: B_TRY(cudaMemcpy(out, b->d_res + b->off_hr(), sizeof(double) * n32, cudaMemcpyDeviceToHost)); return HVP_OK;
        case HVP_OUT_T:
        case HVP_OUT_OMEGA: {
            size_t o = 0;
            for (auto& C : b->circ) {
                B_TRY(cudaMemcpy(out + o, what == HVP_OUT_T ? (const void*)C.T : (const void*)C.Om,
                                 sizeof(double2) * C.ns_real, cudaMemcpyDeviceToHost));
                o += 2 * (size_t)C.ns_real;
            }
            return HVP_OK;
        }
        default: err = "batch: output not available for a batch context"; return HVP_EINVAL;
    }
}

void batch_info(const BatchImpl* b, long long* info) {
    info[0] = b->sumK;
    info[1] = b->n_items;
    info[2] = b->window;
    info[3] = 1;
    info[4] = b->launches;
    info[5] = (long long)(b->bytes >> 20);
    info[6] = b->grid;
    info[7] = b->nc;
    info[8] = kBT;
    info[9] = 1;
}

// Test of the bounded waits: with dep_bias = 1 every chain wait asks for one
// more finished phase than will ever finish, so the first wait runs out after
// spin_limit sleeps and the call reports HVP_ETIMEOUT. The captured graphs
// hold the old values and are dropped.
int batch_wait_test(BatchImpl* b, int dep_bias, long long spin_limit) {
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto& g : b->gexec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    b->dep_bias = dep_bias;
    b->spin_limit = spin_limit;
    return HVP_OK;
}

void batch_free(BatchImpl* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto& g : b->gexec)
        if (g) cudaGraphExecDestroy(g);
    for (void* p : b->allocs) cudaFree(p);
    if (b->h_in) cudaFreeHost(b->h_in);
    if (b->h_res) cudaFreeHost(b->h_res);
    if (b->h_flags) cudaFreeHost(b->h_flags);
    delete b;
}

}  // namespace hvp
