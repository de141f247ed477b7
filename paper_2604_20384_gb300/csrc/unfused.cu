// Unfused sweep: one kernel launch per gate on states in the standard layout
// (qubit 0 = most significant bit). This is the plain schedule of Alg. 1: every
// gate reads and writes its states in HBM. It runs in FP64 (complex128 path)
// or FP32 and serves as the baseline that the window passes are measured
// against.
//
// Forward gate k:  dpsi <- G_k dpsi + V_k psi, psi <- G_k psi   (Eq. dfis, fis)
// Backward gate k: psi^[k-1] = G_k^-1 psi^[k], dpsi^[k-1] = G_k^-1 (dpsi^[k] - V_k psi^[k-1]),
//   environment sums with (a, b) = (phi^[K-k], dphi^[K-k]) (Eq. environment,
//   Eq. Dpsi), then b <- G^dag b + V^dag a, a <- G^dag a (Eq. dbis, bis).
#include "internal.h"

namespace hvp {

namespace {

template <typename R>
struct Cx;
template <>
struct Cx<float> { using T = float2; };
template <>
struct Cx<double> { using T = double2; };

template <typename C>
__device__ __forceinline__ void cmac(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

template <typename C>
__device__ __forceinline__ void cmac_conj(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

template <typename C>
__device__ __forceinline__ C czero() {
    C r;
    r.x = 0;
    r.y = 0;
    return r;
}

__device__ __forceinline__ size_t insert0z(size_t x, int p) {
    return ((x >> p) << (p + 1)) | (x & (((size_t)1 << p) - 1));
}

template <typename C>
struct PairC { C s, t; };  // state and its tangent

template <typename R>
struct MatsR;
template <>
struct MatsR<float> { using T = Mats32; };
template <>
struct MatsR<double> { using T = Mats64; };

template <typename C>
__device__ __forceinline__ void matvec4(const C* M, const C (&x)[4], C (&y)[4]) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        C acc = czero<C>();
#pragma unroll
        for (int c = 0; c < 4; ++c) cmac(acc, M[r * 4 + c], x[c]);
        y[r] = acc;
    }
}

// Four amplitude offsets of gate (q, q+1) for group index alpha.
__device__ __forceinline__ void group_index(size_t alpha, int n, int q, size_t (&idx)[4]) {
    const int phi = n - 1 - q, plo = n - 2 - q;  // bits of qubit q and q + 1
    const size_t l0 = insert0z(insert0z(alpha, plo), phi);
    idx[0] = l0;
    idx[1] = l0 | ((size_t)1 << plo);
    idx[2] = l0 | ((size_t)1 << phi);
    idx[3] = idx[1] | ((size_t)1 << phi);
}

template <typename R, bool TAN>
__global__ void u_init_kernel(const typename Cx<R>::T* __restrict__ psi1q, void* xv, int n, int ns) {
    using C = typename Cx<R>::T;
    const size_t dim = (size_t)1 << n;
    const size_t total = dim * ns;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t s = i >> n, x = i & (dim - 1);
        C amp;
        amp.x = 1;
        amp.y = 0;
        for (int q = 0; q < n; ++q) amp = cmul(amp, psi1q[(s * n + q) * 2 + ((x >> (n - 1 - q)) & 1)]);
        if constexpr (TAN) {
            reinterpret_cast<PairC<C>*>(xv)[i] = PairC<C>{amp, czero<C>()};
        } else {
            reinterpret_cast<C*>(xv)[i] = amp;
        }
    }
}

template <typename R, bool TAN>
__global__ void u_load_phi_kernel(const typename Cx<R>::T* __restrict__ phi, void* cv, size_t total) {
    using C = typename Cx<R>::T;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        if constexpr (TAN) reinterpret_cast<PairC<C>*>(cv)[i] = PairC<C>{phi[i], czero<C>()};
        else reinterpret_cast<C*>(cv)[i] = phi[i];
    }
}

template <typename R, bool TAN>
__global__ void u_fwd_kernel(const typename MatsR<R>::T* __restrict__ mats, int k, int q, void* xv, int n, int ns) {
    using C = typename Cx<R>::T;
    const C* G = mats[k].G;
    const C* V = mats[k].V;
    const size_t groups = (size_t)1 << (n - 2);
    const size_t total = groups * ns;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t s = i / groups, alpha = i - s * groups;
        size_t idx[4];
        group_index(alpha, n, q, idx);
        const size_t off = s << n;
        if constexpr (TAN) {
            PairC<C>* x = reinterpret_cast<PairC<C>*>(xv) + off;
            C p[4], d[4], np[4], nd[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) { p[c] = x[idx[c]].s; d[c] = x[idx[c]].t; }
            matvec4(G, p, np);
            matvec4(G, d, nd);
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) cmac(nd[r], V[r * 4 + c], p[c]);
#pragma unroll
            for (int r = 0; r < 4; ++r) x[idx[r]] = PairC<C>{np[r], nd[r]};
        } else {
            C* x = reinterpret_cast<C*>(xv) + off;
            C p[4], np[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) p[c] = x[idx[c]];
            matvec4(G, p, np);
#pragma unroll
            for (int r = 0; r < 4; ++r) x[idx[r]] = np[r];
        }
    }
}

constexpr int kUT = 256;  // threads of the unfused backward kernel

template <typename R, bool TAN>
__global__ void __launch_bounds__(kUT) u_bwd_kernel(const typename MatsR<R>::T* __restrict__ mats, int k, int q,
                                                    void* xv, void* cv, double* __restrict__ partial, int n, int ns,
                                                    int cx_count) {
    using C = typename Cx<R>::T;
    constexpr int NE = TAN ? 32 : 16;   // complex components: E then DE
    __shared__ double sred[kUT / 32][2 * NE];
    const C* Gi = mats[k].Ginv;
    const C* Gh = mats[k].Gh;
    const C* V = mats[k].V;
    const C* Vh = mats[k].Vh;
    const int s = blockIdx.y;
    const size_t groups = (size_t)1 << (n - 2);
    const size_t per = (groups + cx_count - 1) / cx_count;
    const size_t g0 = blockIdx.x * per, g1 = min(groups, g0 + per);
    const size_t off = (size_t)s << n;
    C red[NE];
#pragma unroll
    for (int e = 0; e < NE; ++e) red[e] = czero<C>();
    for (size_t alpha = g0 + threadIdx.x; alpha < g1; alpha += kUT) {
        size_t idx[4];
        group_index(alpha, n, q, idx);
        if constexpr (TAN) {
            PairC<C>* x = reinterpret_cast<PairC<C>*>(xv) + off;
            PairC<C>* c = reinterpret_cast<PairC<C>*>(cv) + off;
            // Forward states first (written back before the co-states are
            // loaded), so that fewer values are live beside the 32 complex
            // accumulators: the complex128 form would not fit in registers.
            C pp[4], dp[4], A[4], B[4], nA[4], nB[4];
            {
                C p[4], tt[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) p[j] = x[idx[j]].s;
                matvec4(Gi, p, pp);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    tt[r] = x[idx[r]].t;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        C mv = V[r * 4 + j];
                        mv.x = -mv.x;
                        mv.y = -mv.y;
                        cmac(tt[r], mv, pp[j]);
                    }
                }
                matvec4(Gi, tt, dp);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) x[idx[r]] = PairC<C>{pp[r], dp[r]};
#pragma unroll
            for (int j = 0; j < 4; ++j) { A[j] = c[idx[j]].s; B[j] = c[idx[j]].t; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    cmac_conj(red[i * 4 + j], A[i], pp[j]);
                    cmac_conj(red[16 + i * 4 + j], B[i], pp[j]);
                    cmac_conj(red[16 + i * 4 + j], A[i], dp[j]);
                }
            matvec4(Gh, A, nA);
            matvec4(Gh, B, nB);
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int j = 0; j < 4; ++j) cmac(nB[r], Vh[r * 4 + j], A[j]);
#pragma unroll
            for (int r = 0; r < 4; ++r) c[idx[r]] = PairC<C>{nA[r], nB[r]};
        } else {
            C* x = reinterpret_cast<C*>(xv) + off;
            C* c = reinterpret_cast<C*>(cv) + off;
            C p[4], A[4], pp[4], nA[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) { p[j] = x[idx[j]]; A[j] = c[idx[j]]; }
            matvec4(Gi, p, pp);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cmac_conj(red[i * 4 + j], A[i], pp[j]);
            matvec4(Gh, A, nA);
#pragma unroll
            for (int r = 0; r < 4; ++r) { x[idx[r]] = pp[r]; c[idx[r]] = nA[r]; }
        }
    }
    // Warp tree in the state precision, then FP64 across warps.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < NE; ++e) {
        R vx = red[e].x, vy = red[e].y;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            vx += __shfl_xor_sync(0xffffffffu, vx, o);
            vy += __shfl_xor_sync(0xffffffffu, vy, o);
        }
        if (lane == 0) { sred[warp][2 * e] = (double)vx; sred[warp][2 * e + 1] = (double)vy; }
    }
    __syncthreads();
    if (threadIdx.x < 64) {
        double sum = 0.0;
        if (threadIdx.x < 2 * NE)
            for (int ww = 0; ww < kUT / 32; ++ww) sum += sred[ww][threadIdx.x];
        partial[(((size_t)k * ns + s) * cx_count + blockIdx.x) * 64 + threadIdx.x] = sum;
    }
}

inline int grid_for(size_t total, int threads) {
    size_t b = (total + threads - 1) / threads;
    return (int)(b > 152 * 64 ? 152 * 64 : (b < 1 ? 1 : b));
}

}  // namespace

int unfused_cx_count(int n, int ns) {
    // Enough CTAs per sample to fill 152 SMs several times, at most one CTA
    // per 256 groups of four amplitudes.
    const long long groups = 1ll << (n - 2);
    long long cx = (152 * 8 + ns - 1) / ns;
    long long maxcx = (groups + kUT - 1) / kUT;
    if (cx > maxcx) cx = maxcx;
    if (cx < 1) cx = 1;
    return (int)cx;
}

cudaError_t unfused_init(bool dbl, const void* psi1q, void* x, int n, int ns, bool tan, cudaStream_t st) {
    const size_t total = ((size_t)1 << n) * ns;
    const int gr = grid_for(total, 256);
    if (dbl) {
        if (tan) u_init_kernel<double, true><<<gr, 256, 0, st>>>((const double2*)psi1q, x, n, ns);
        else u_init_kernel<double, false><<<gr, 256, 0, st>>>((const double2*)psi1q, x, n, ns);
    } else {
        if (tan) u_init_kernel<float, true><<<gr, 256, 0, st>>>((const float2*)psi1q, x, n, ns);
        else u_init_kernel<float, false><<<gr, 256, 0, st>>>((const float2*)psi1q, x, n, ns);
    }
    return cudaGetLastError();
}

cudaError_t unfused_load_phi(bool dbl, const void* phi, void* c, int n, int ns, bool tan, cudaStream_t st) {
    const size_t total = ((size_t)1 << n) * ns;
    const int gr = grid_for(total, 256);
    if (dbl) {
        if (tan) u_load_phi_kernel<double, true><<<gr, 256, 0, st>>>((const double2*)phi, c, total);
        else u_load_phi_kernel<double, false><<<gr, 256, 0, st>>>((const double2*)phi, c, total);
    } else {
        if (tan) u_load_phi_kernel<float, true><<<gr, 256, 0, st>>>((const float2*)phi, c, total);
        else u_load_phi_kernel<float, false><<<gr, 256, 0, st>>>((const float2*)phi, c, total);
    }
    return cudaGetLastError();
}

cudaError_t unfused_fwd_gate(bool dbl, const void* mats, int k, int q, void* x, int n, int ns, bool tan,
                             cudaStream_t st) {
    const size_t total = ((size_t)1 << (n - 2)) * ns;
    const int gr = grid_for(total, 256);
    if (dbl) {
        if (tan) u_fwd_kernel<double, true><<<gr, 256, 0, st>>>((const Mats64*)mats, k, q, x, n, ns);
        else u_fwd_kernel<double, false><<<gr, 256, 0, st>>>((const Mats64*)mats, k, q, x, n, ns);
    } else {
        if (tan) u_fwd_kernel<float, true><<<gr, 256, 0, st>>>((const Mats32*)mats, k, q, x, n, ns);
        else u_fwd_kernel<float, false><<<gr, 256, 0, st>>>((const Mats32*)mats, k, q, x, n, ns);
    }
    return cudaGetLastError();
}

cudaError_t unfused_bwd_gate(bool dbl, const void* mats, int k, int q, void* x, void* c, double* partial, int n,
                             int ns, int cx_count, bool tan, cudaStream_t st) {
    dim3 grid(cx_count, ns);
    if (dbl) {
        if (tan) u_bwd_kernel<double, true><<<grid, kUT, 0, st>>>((const Mats64*)mats, k, q, x, c, partial, n, ns, cx_count);
        else u_bwd_kernel<double, false><<<grid, kUT, 0, st>>>((const Mats64*)mats, k, q, x, c, partial, n, ns, cx_count);
    } else {
        if (tan) u_bwd_kernel<float, true><<<grid, kUT, 0, st>>>((const Mats32*)mats, k, q, x, c, partial, n, ns, cx_count);
        else u_bwd_kernel<float, false><<<grid, kUT, 0, st>>>((const Mats32*)mats, k, q, x, c, partial, n, ns, cx_count);
    }
    return cudaGetLastError();
}

}  // namespace hvp
