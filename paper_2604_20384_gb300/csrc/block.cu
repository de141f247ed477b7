// FP64 parts of the fused-block (tensor-core) schedule: per-call block
// operators, the overlaps that weight the co-states, and the reduction of
// block environments to per-gate gradient and HVP blocks.
//
// A block j holds the gates G_1 .. G_m (circuit order) that act inside the
// five qubits [a, a + 5); its index b has qubit a + i on bit 4 - i. With
// every gate embedded in the block (identity on the other three qubits),
//     B = G_m ... G_1,      dB = sum_i G_m .. V_i .. G_1      (App. D: the
// tangent of a product is the block-triangular operator [[B, 0], [dB, B]]).
// The tensor-core passes apply [[B, 0], [dB, B]] forward to (psi, dpsi) and
// [[B^dag, 0], [dB^dag, B^dag]] backward to the co-states (c, dc) as one real
// GEMM per tile: the 128 x 64 operator B over dB times the columns psi | dpsi
// gives B psi, B dpsi over dB psi, dB dpsi, of which psi' = B psi and dpsi' =
// B dpsi + dB psi are read (likewise backward). The operator is stored as
// three slices of 8-bit integers per row (see internal.h).
//
// Block environments. The backward pass accumulates, over every amplitude
// of every sample, P[4a + p][4b + q] = sum C_p[a] Psi_q[b], where C = (re c,
// im c, re dc, im dc) are the co-states at the block's input (after the
// block's backward update) and Psi the forward states there. With
//     Y_0  = sum conj(c) psi^T,   dY_0 = sum conj(dc) psi^T + conj(c) dpsi^T
// read off P, the gates i = 1 .. m of the block follow by moving the cut one
// gate at a time (Eq. bis: c before gate i = G_i^dag c after it):
//     Ehat_i  = G_i^-T Y_{i-1},          E_i  = ptr Ehat_i,
//     dEhat_i = G_i^-T dY_{i-1} - Y_i^T Y_{i-1},   DE_i = ptr dEhat_i,
//     Y_i     = Ehat_i G_i^T,            dY_i = dEhat_i G_i^T + Ehat_i V_i^T,
// where Y_i = G_i^-1 V_i G_i^-1 is the derivative of G_i^-1 (up to sign),
// Ehat_i = sum conj(c after gate i) (psi before gate i)^T is Eq. environment
// before the partial trace ptr over the block's three other qubits, and
// dEhat_i its derivative along V (Eq. Dpsi). The co-states enter
// pre-weighted by the overlaps, (T_s phi_s, Omega_s phi_s), so these sums are
// already sum_s conj(T_s) E_s and sum_s (conj(Omega_s) E_s + conj(T_s) DE_s),
// the quantities of Eq. grad-costHS and Eq. hvp-costHS (with the sign
// reading of Eq. costHS); the Frobenius cost starts from (phi_s, 0).
#include "internal.h"

namespace hvp {

namespace {

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }

// The four block indices of a gate acting on bits (hb, lb = hb - 1) of the
// block index, the other three bits taken from x: r[2i + j] has bit hb = i
// and bit lb = j.
__device__ __forceinline__ void gate_rows(int x, int hb, int (&r)[4]) {
    const int lb = hb - 1;
    const int low = x & ((1 << lb) - 1);
    const int r0 = ((x >> lb) << (hb + 1)) | low;
    r[0] = r0;
    r[1] = r0 | (1 << lb);
    r[2] = r0 | (1 << hb);
    r[3] = r0 | (1 << hb) | (1 << lb);
}

// Real embedding of a complex entry x: output component qr (re, im) from
// input component qc (re, im).
__device__ __forceinline__ double embed(int qr, int qc, double2 x) {
    return qr == 0 ? (qc == 0 ? x.x : -x.y) : (qc == 0 ? x.y : x.x);
}

// bf16 bits of an integer of magnitude <= 256 (exact).
__device__ __forceinline__ uint32_t bf16_int(double v) { return __float_as_uint((float)v) >> 16; }

// One CTA per block (256 threads): B and dB by applying the block's gates to
// the identity, then the block's operator record (see internal.h): for each
// direction, each of the 128 rows (B over dB) is split into three slices of
// 8-bit integers on a common power-of-two row scale, so that the tensor-core
// products of slices and their sums over K = 64 are exact integers in FP32.
__global__ void __launch_bounds__(256) block_prep_kernel(const DevBlock* __restrict__ blocks,
                                                          const DevBlockGate* __restrict__ bg,
                                                          const double2* __restrict__ G,
                                                          const double2* __restrict__ V, uint32_t* __restrict__ ops,
                                                          int* status) {
    __shared__ double2 M[32 * 32], dM[32 * 32];
    __shared__ double2 sg[16], sv[16];
    const DevBlock blk = blocks[blockIdx.x];
    const int t = threadIdx.x, col = t & 31, x = t >> 5;
    for (int e = t; e < 1024; e += 256) {
        M[e] = make_double2((e >> 5) == (e & 31) ? 1.0 : 0.0, 0.0);
        dM[e] = make_double2(0.0, 0.0);
    }
    bool ok = true;
    for (int i = 0; i < blk.n_gates; ++i) {
        const DevBlockGate g = bg[blk.gate_off + i];
        __syncthreads();
        if (t < 16) {
            sg[t] = G[(size_t)g.k * 16 + t];
            sv[t] = V ? V[(size_t)g.k * 16 + t] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        int r[4];
        gate_rows(x, 4 - g.u, r);
        double2 m[4], dm[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            m[c] = M[r[c] * 32 + col];
            dm[c] = dM[r[c] * 32 + col];
        }
        __syncthreads();
#pragma unroll
        for (int rw = 0; rw < 4; ++rw) {
            double2 a = make_double2(0.0, 0.0), d = make_double2(0.0, 0.0);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                a = zadd(a, zmul(sg[rw * 4 + c], m[c]));
                d = zadd(d, zadd(zmul(sg[rw * 4 + c], dm[c]), zmul(sv[rw * 4 + c], m[c])));
            }
            M[r[rw] * 32 + col] = a;
            dM[r[rw] * 32 + col] = d;
        }
    }
    __syncthreads();
    uint32_t* o = ops + (size_t)blockIdx.x * kOpWords;
    float* scales = reinterpret_cast<float*>(o + kOpScaleOff);
    // 256 (direction, row) lines, one per thread: rows 2 b' + q of X (B or
    // B^dag), then 64 + 2 b' + q of dX; entries K = 2 b + (re, im).
    {
        const int line = t, d = line >> 7, row = line & 127, b1 = (row & 63) >> 1, q1 = row & 1;
        const bool drow = row >= 64;
        auto entry = [&](int k) {
            const int b0 = k >> 1;
            const double2 m = drow ? (d ? zconj(dM[b0 * 32 + b1]) : dM[b1 * 32 + b0])
                                   : (d ? zconj(M[b0 * 32 + b1]) : M[b1 * 32 + b0]);
            return embed(q1, k & 1, m);
        };
        double amax = 0.0;
        for (int k = 0; k < 64; ++k) {
            const double v = entry(k);
            ok = ok && isfinite(v);
            amax = fmax(amax, fabs(v));
        }
        int f = 0;
        if (amax > 0.0 && isfinite(amax)) frexp(amax, &f);   // 2^f > amax >= 2^(f-1)
        const double up = ldexp(1.0, 8 - f);
        scales[d * 128 + row] = (float)ldexp(1.0, f - 8);
        uint32_t* s0 = o + (d * 3 + 0) * kOpSliceWords + row * 32;
        uint32_t* s1 = s0 + kOpSliceWords;
        uint32_t* s2 = s1 + kOpSliceWords;
        for (int w = 0; w < 32; ++w) {
            uint32_t q0 = 0, qa = 0, qb = 0;
            for (int hlf = 0; hlf < 2; ++hlf) {
                const double y = isfinite(amax) ? entry(2 * w + hlf) * up : 0.0;
                const double a0 = rint(y), y1 = (y - a0) * 256.0, a1 = rint(y1), a2 = rint((y1 - a1) * 256.0);
                q0 |= bf16_int(a0) << (16 * hlf);
                qa |= bf16_int(a1) << (16 * hlf);
                qb |= bf16_int(a2) << (16 * hlf);
            }
            s0[w] = q0;
            s1[w] = qa;
            s2[w] = qb;
        }
    }
    if (!ok) atomicOr(status, 1);
}

// T_s = sum conj(phi_s) psi_s^[K], Omega_s = sum conj(phi_s) dpsi_s^[K]
// (Eq. overlap-general at the end of the circuit; Eq. Omega as phi^dag dpsi),
// per (sample, chunk) partial sums: FP32 runs of 8 amplitudes summed in FP64.
__global__ void __launch_bounds__(256) overlap_partial_kernel(const float4* __restrict__ x,
                                                               const float2* __restrict__ phi, double* partial,
                                                               int n, int chunks) {
    const int s = blockIdx.y, t = threadIdx.x;
    const size_t dim = (size_t)1 << n, per = (dim + chunks - 1) / chunks;
    const size_t lo = per * blockIdx.x, hi = min(dim, lo + per);
    // FP32 fused multiply-adds over runs of 8 amplitudes, each run's sums
    // added in FP64 (FP64 arithmetic is a small fraction of the FP32 rate).
    double tr = 0, ti = 0, orr = 0, oi = 0;
    for (size_t i = lo + t; i < hi;) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k, i += 256) {
            if (i < hi) {
                const float4 v = __ldcs(&x[(size_t)s * dim + i]);
                const float2 p = __ldg(&phi[(size_t)s * dim + i]);
                a0 = fmaf(p.x, v.x, fmaf(p.y, v.y, a0));
                a1 = fmaf(p.x, v.y, fmaf(-p.y, v.x, a1));
                a2 = fmaf(p.x, v.z, fmaf(p.y, v.w, a2));
                a3 = fmaf(p.x, v.w, fmaf(-p.y, v.z, a3));
            }
        }
        tr += (double)a0;
        ti += (double)a1;
        orr += (double)a2;
        oi += (double)a3;
    }
    __shared__ double sh[4][256];
    sh[0][t] = tr; sh[1][t] = ti; sh[2][t] = orr; sh[3][t] = oi;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w)
            for (int q = 0; q < 4; ++q) sh[q][t] += sh[q][t + w];
        __syncthreads();
    }
    if (t < 4) partial[((size_t)s * chunks + blockIdx.x) * 4 + t] = sh[t][0];
}

__global__ void overlap_final_kernel(const double* __restrict__ partial, double2* T, double2* Om, int ns,
                                     int chunks) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    double q[4] = {0, 0, 0, 0};
    for (int c = 0; c < chunks; ++c)
        for (int i = 0; i < 4; ++i) q[i] += partial[((size_t)s * chunks + c) * 4 + i];
    T[s] = make_double2(q[0], q[1]);
    Om[s] = make_double2(q[2], q[3]);
}

// P summed over the per-CTA FP64 records, in a fixed order: sum[j][e] =
// sum_c rec[j][c][e].
__global__ void block_env_reduce_kernel(const double* __restrict__ rec, double* __restrict__ sum, int nb, int cx) {
    const size_t total = (size_t)nb * 16384;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t j = i >> 14, e = i & 16383;
        const double* src = rec + j * (size_t)cx * 16384 + e;
        double a = 0.0;
        for (int c = 0; c < cx; ++c) a += src[(size_t)c * 16384];
        sum[i] = a;
    }
}

// One CTA per block (256 threads): per-gate weighted environments E_i, DE_i
// from the block's P by the recursion of the file header.
__global__ void __launch_bounds__(256) block_post_kernel(const DevBlock* __restrict__ blocks,
                                                          const DevBlockGate* __restrict__ bg,
                                                          const double* __restrict__ P,
                                                          const Mats64* __restrict__ mats, double2* Ew,
                                                          double2* DEw, int tangent) {
    __shared__ double2 Yc[32 * 32], dYc[32 * 32];   // Y_{i-1}, then Ehat_i, then Y_i (in place)
    __shared__ double2 sGt[16], sGi[16], sYt[16], sV[16];
    const DevBlock blk = blocks[blockIdx.x];
    const double* Pj = P + (size_t)blockIdx.x * 16384;
    const int t = threadIdx.x;
    for (int e = t; e < 1024; e += 256) {
        const int a = e >> 5, b = e & 31;
        auto p = [&](int pa, int pb) { return Pj[(4 * a + pa) * 128 + 4 * b + pb]; };
        Yc[e] = make_double2(p(0, 0) + p(1, 1), p(0, 1) - p(1, 0));
        dYc[e] = tangent ? make_double2(p(2, 0) + p(3, 1) + p(0, 2) + p(1, 3), p(2, 1) - p(3, 0) + p(0, 3) - p(1, 2))
                         : make_double2(0.0, 0.0);
    }
    for (int i = 0; i < blk.n_gates; ++i) {
        const DevBlockGate g = bg[blk.gate_off + i];
        const Mats64& mg = mats[g.k];
        const int hb = 4 - g.u;
        if (t < 16) {
            sGi[t] = mg.Ginv[t];
            sGt[t] = mg.G[t];
            sYt[t] = tangent ? mg.Y[t] : make_double2(0.0, 0.0);
            sV[t] = tangent ? mg.V[t] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        // Ehat = G^-T Y ; dEhat = G^-T dY - Y_g^T Y
        {
            const int col = t & 31, x = t >> 5;
            int r[4];
            gate_rows(x, hb, r);
            double2 y[4], dy[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                y[c] = Yc[r[c] * 32 + col];
                dy[c] = dYc[r[c] * 32 + col];
            }
            double2 a[4], d[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = make_double2(0.0, 0.0);
                d[q] = make_double2(0.0, 0.0);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    a[q] = zadd(a[q], zmul(sGi[k * 4 + q], y[k]));
                    d[q] = zadd(d[q], zmul(sGi[k * 4 + q], dy[k]));
                    const double2 w = zmul(sYt[k * 4 + q], y[k]);
                    d[q] = make_double2(d[q].x - w.x, d[q].y - w.y);
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                Yc[r[q] * 32 + col] = a[q];
                dYc[r[q] * 32 + col] = d[q];
            }
        }
        __syncthreads();
        // E_i[c][d] = sum_x Ehat[(c,x)][(d,x)] (partial trace over the other three qubits)
        if (t < 32) {
            const int e = t & 15, which = t >> 4, c = e >> 2, d = e & 3;
            const double2* S = which ? dYc : Yc;
            double2 acc = make_double2(0.0, 0.0);
            for (int x = 0; x < 8; ++x) {
                int rr[4];
                gate_rows(x, hb, rr);
                acc = zadd(acc, S[rr[c] * 32 + rr[d]]);
            }
            if (which == 0) Ew[(size_t)g.k * 16 + e] = acc;
            else DEw[(size_t)g.k * 16 + e] = tangent ? acc : make_double2(0.0, 0.0);
        }
        if (i + 1 == blk.n_gates) break;
        // Y <- Ehat G^T ; dY <- dEhat G^T + Ehat V^T   (right multiplication on column bits)
        {
            const int row = t & 31, x = t >> 5;
            int c4[4];
            gate_rows(x, hb, c4);
            double2 e4[4], de4[4], a[4], d[4];
            __syncthreads();   // the partial traces above have read Ehat
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                e4[k] = Yc[row * 32 + c4[k]];
                de4[k] = dYc[row * 32 + c4[k]];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = make_double2(0.0, 0.0);
                d[q] = make_double2(0.0, 0.0);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    a[q] = zadd(a[q], zmul(e4[k], sGt[q * 4 + k]));
                    d[q] = zadd(d[q], zadd(zmul(de4[k], sGt[q * 4 + k]), zmul(e4[k], sV[q * 4 + k])));
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                Yc[row * 32 + c4[q]] = a[q];
                dYc[row * 32 + c4[q]] = d[q];
            }
        }
        __syncthreads();
    }
}

// The states (first two components) of float4 (psi, dpsi) elements.
__global__ void extract_psi_kernel(const float4* __restrict__ x, float2* __restrict__ out, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const float4 v = x[i];
        out[i] = make_float2(v.x, v.y);
    }
}

// The product input states psi^[0]_s = (x)_q psi_{s,q} (Eq. costHS) as
// float4 (psi, dpsi = 0), factors multiplied in qubit order.
__global__ void product_states_kernel(const float2* __restrict__ q1, float4* __restrict__ out, int n, size_t count) {
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < count; g += (size_t)gridDim.x * blockDim.x) {
        const size_t s = g >> n;
        const unsigned long long idx = g & ((1ull << n) - 1ull);
        const float2* f = q1 + s * (size_t)n * 2;
        float2 a = make_float2(1.f, 0.f);
        for (int q = 0; q < n; ++q) {
            const float2 v = __ldg(&f[2 * q + ((idx >> (n - 1 - q)) & 1ull)]);
            a = make_float2(a.x * v.x - a.y * v.y, a.x * v.y + a.y * v.x);
        }
        out[g] = make_float4(a.x, a.y, 0.f, 0.f);
    }
}

// The co-states entering the backward sweep, weighted by the overlaps:
// (w1_s phi_s, w2_s phi_s), w1 = T_s and w2 = Omega_s (or 1 and 0 when null).
__global__ void weighted_phi_kernel(const float2* __restrict__ phi, const double2* __restrict__ w1,
                                    const double2* __restrict__ w2, float4* __restrict__ out, int n, size_t count) {
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < count; g += (size_t)gridDim.x * blockDim.x) {
        const float2 ph = __ldg(&phi[g]);
        const size_t s = g >> n;
        float2 a = make_float2(1.f, 0.f), b = make_float2(0.f, 0.f);
        if (w1) a = make_float2((float)w1[s].x, (float)w1[s].y);
        if (w2) b = make_float2((float)w2[s].x, (float)w2[s].y);
        out[g] = make_float4(a.x * ph.x - a.y * ph.y, a.x * ph.y + a.y * ph.x, b.x * ph.x - b.y * ph.y,
                             b.x * ph.y + b.y * ph.x);
    }
}

}  // namespace

cudaError_t launch_product_states(const float2* psi1q, float4* out, int n, int ns, cudaStream_t st) {
    const size_t count = ((size_t)1 << n) * ns;
    size_t blocks = (count + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    product_states_kernel<<<(int)blocks, 256, 0, st>>>(psi1q, out, n, count);
    return cudaGetLastError();
}

cudaError_t launch_weighted_phi(const float2* phi, const double2* w1, const double2* w2, float4* out, int n, int ns,
                                cudaStream_t st) {
    const size_t count = ((size_t)1 << n) * ns;
    size_t blocks = (count + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    weighted_phi_kernel<<<(int)blocks, 256, 0, st>>>(phi, w1, w2, out, n, count);
    return cudaGetLastError();
}

cudaError_t launch_extract_psi(const float4* x, float2* out, size_t count, cudaStream_t st) {
    size_t blocks = (count + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    extract_psi_kernel<<<(int)blocks, 256, 0, st>>>(x, out, count);
    return cudaGetLastError();
}

cudaError_t launch_block_prep(const DevBlock* blocks, const DevBlockGate* bg, int nb, const double2* G,
                              const double2* V, uint32_t* ops, int* status, cudaStream_t st) {
    block_prep_kernel<<<nb, 256, 0, st>>>(blocks, bg, G, V, ops, status);
    return cudaGetLastError();
}

cudaError_t launch_overlaps(const float4* x, const float2* phi, double* partial, double2* T, double2* Om, int n,
                            int ns, int chunks, cudaStream_t st) {
    overlap_partial_kernel<<<dim3(chunks, ns), 256, 0, st>>>(x, phi, partial, n, chunks);
    overlap_final_kernel<<<(ns + 127) / 128, 128, 0, st>>>(partial, T, Om, ns, chunks);
    return cudaGetLastError();
}

cudaError_t launch_block_post(const DevBlock* blocks, const DevBlockGate* bg, int nb, const double* rec, int cx,
                              double* psum, const Mats64* mats, double2* Ew, double2* DEw, int tangent,
                              cudaStream_t st) {
    block_env_reduce_kernel<<<152 * 4, 256, 0, st>>>(rec, psum, nb, cx);
    block_post_kernel<<<nb, 256, 0, st>>>(blocks, bg, psum, mats, Ew, DEw, tangent);
    return cudaGetLastError();
}

}  // namespace hvp
