// FP64 kernels around the sweeps: per-call gate preparation, reduction of the
// per-CTA environment records, the overlaps T_s and Omega_s, the loss, the
// gradient and HVP of the sampled cost (Alg. 2 with the sign reading of
// Eq. costHS) and their Riemannian forms (App. F). All of it is a few kB of
// data; it runs in FP64 on the GPU so that no result leaves the device
// before it is final.
#include "internal.h"

namespace hvp {

namespace {

__device__ __forceinline__ double2 dmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 dadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 dsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 dconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 dscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ bool dfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// G^-1, G^dag, V^dag per gate; Gauss-Jordan elimination with partial pivoting
// in FP64. A singular or non-finite gate sets status bit 1.
template <typename MT, typename C>
__device__ void store_mats(MT& m, const double2 (&G)[16], const double2 (&Gi)[16], const double2 (&V)[16],
                           const double2 (&Y)[16]) {
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            const int e = r * 4 + c;
            C g, gi, gh, v, vh;
            g.x = G[e].x; g.y = G[e].y;
            gi.x = Gi[e].x; gi.y = Gi[e].y;
            gh.x = G[c * 4 + r].x; gh.y = -G[c * 4 + r].y;
            v.x = V[e].x; v.y = V[e].y;
            vh.x = V[c * 4 + r].x; vh.y = -V[c * 4 + r].y;
            C y;
            y.x = Y[e].x; y.y = Y[e].y;
            m.G[e] = g; m.Ginv[e] = gi; m.Gh[e] = gh; m.V[e] = v; m.Vh[e] = vh; m.Y[e] = y;
        }
}

__global__ void prep_kernel(const double2* __restrict__ Gin, const double2* __restrict__ Vin, void* mats, int dbl,
                            int K, int* status) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    double2 G[16], V[16], A[4][8];
    bool ok = true;
    for (int e = 0; e < 16; ++e) {
        G[e] = Gin[k * 16 + e];
        V[e] = Vin ? Vin[k * 16 + e] : make_double2(0.0, 0.0);
        ok = ok && dfinite(G[e]) && dfinite(V[e]);
    }
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 8; ++c) A[r][c] = c < 4 ? G[r * 4 + c] : make_double2(c - 4 == r ? 1.0 : 0.0, 0.0);
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        double best = -1.0;
        for (int r = col; r < 4; ++r) {
            const double m = A[r][col].x * A[r][col].x + A[r][col].y * A[r][col].y;
            if (m > best) { best = m; piv = r; }
        }
        if (!(best > 0.0)) { ok = false; break; }
        if (piv != col)
            for (int c = 0; c < 8; ++c) { double2 t = A[col][c]; A[col][c] = A[piv][c]; A[piv][c] = t; }
        const double2 p = A[col][col];
        const double den = p.x * p.x + p.y * p.y;
        const double2 ip = make_double2(p.x / den, -p.y / den);
        for (int c = 0; c < 8; ++c) A[col][c] = dmul(A[col][c], ip);
        for (int r = 0; r < 4; ++r) {
            if (r == col) continue;
            const double2 f = A[r][col];
            for (int c = 0; c < 8; ++c) A[r][c] = dsub(A[r][c], dmul(f, A[col][c]));
        }
    }
    double2 Gi[16];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            Gi[r * 4 + c] = A[r][c + 4];
            ok = ok && dfinite(Gi[r * 4 + c]);
        }
    if (!ok) atomicOr(status, 1);
    double2 GV[16], Y[16];                       // Y = G^-1 V G^-1
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double2 a = make_double2(0.0, 0.0);
            for (int t = 0; t < 4; ++t) a = dadd(a, dmul(Gi[r * 4 + t], V[t * 4 + c]));
            GV[r * 4 + c] = a;
        }
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double2 a = make_double2(0.0, 0.0);
            for (int t = 0; t < 4; ++t) a = dadd(a, dmul(GV[r * 4 + t], Gi[t * 4 + c]));
            Y[r * 4 + c] = a;
        }
    if (dbl) store_mats<Mats64, double2>(reinterpret_cast<Mats64*>(mats)[k], G, Gi, V, Y);
    else store_mats<Mats32, float2>(reinterpret_cast<Mats32*>(mats)[k], G, Gi, V, Y);
}

// env[s][k][e] = sum over CTAs of partial[k][s][cx][e]; one warp per (k, s).
__global__ void reduce_kernel(const double* __restrict__ partial, double* __restrict__ env, int K, int ns, int cx) {
    const int pair = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (pair >= K * ns) return;
    const int k = pair / ns, s = pair - k * ns;
    const double* src = partial + ((size_t)k * ns + s) * cx * 64;
    double a0 = 0.0, a1 = 0.0;
    for (int c = 0; c < cx; ++c) {
        a0 += src[(size_t)c * 64 + lane];
        a1 += src[(size_t)c * 64 + lane + 32];
    }
    double* dst = env + ((size_t)s * K + k) * 64;
    dst[lane] = a0;
    dst[lane + 32] = a1;
}

// T_s = sum_ij (dT_s/dG_K)_ij (G_K)_ij (Eq. overlap-2 at the last gate) and
// Omega_s = sum_k sum_ij (dT_s/dG_k)_ij (V_k)_ij (Eq. Omega, App. B).
__global__ void overlaps_kernel(const double* __restrict__ env, const double2* __restrict__ G,
                                const double2* __restrict__ V, double2* T, double2* Om, int K, int tangent) {
    const int s = blockIdx.x;
    __shared__ double2 sh[256];
    const double2* Es = reinterpret_cast<const double2*>(env + (size_t)s * K * 64);
    double2 om = make_double2(0.0, 0.0);
    if (tangent)
        for (int i = threadIdx.x; i < K * 16; i += blockDim.x) {
            const int k = i >> 4, e = i & 15;
            om = dadd(om, dmul(Es[k * 32 + e], V[k * 16 + e]));
        }
    sh[threadIdx.x] = om;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = dadd(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double2 t = make_double2(0.0, 0.0);
        for (int e = 0; e < 16; ++e) t = dadd(t, dmul(Es[(K - 1) * 32 + e], G[(K - 1) * 16 + e]));
        T[s] = t;
        Om[s] = tangent ? sh[0] : make_double2(0.0, 0.0);
    }
}

// Stores gate k's entry e (16 threads per gate) of the Euclidean gradient g
// and HVP h, then their projections to the tangent space of U(4) at G_k
// (App. F): grad_R = P_G(g), H_R = P_G(h - V g^dag G / 2 - G g^dag V / 2),
// with P_G(X) = X / 2 - G X^dag G / 2.
__device__ void finish_gate(int k, int e, double2 g, double2 h, const double2* __restrict__ G,
                            const double2* __restrict__ V, double2* ge, double2* he, double2* gr, double2* hr,
                            int tangent) {
    __shared__ double2 sG[16], sV[16], sg[16], sX[16];
    sG[e] = G[k * 16 + e];
    sV[e] = tangent ? V[k * 16 + e] : make_double2(0.0, 0.0);
    sg[e] = g;
    ge[k * 16 + e] = g;
    if (tangent) he[k * 16 + e] = h;
    __syncthreads();
    const int r = e >> 2, c = e & 3;
    // A B^dag C entry (r, c) = sum_a sum_b A[r][a] conj(B[b][a]) C[b][c].
    auto abdc = [&](const double2* A, const double2* B, const double2* Cm) {
        double2 acc = make_double2(0.0, 0.0);
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) acc = dadd(acc, dmul(dmul(A[r * 4 + a], dconj(B[b * 4 + a])), Cm[b * 4 + c]));
        return acc;
    };
    gr[k * 16 + e] = dsub(dscale(g, 0.5), dscale(abdc(sG, sg, sG), 0.5));
    if (tangent) {
        const double2 x = dsub(dsub(h, dscale(abdc(sV, sg, sG), 0.5)), dscale(abdc(sG, sg, sV), 0.5));
        sX[e] = x;
        __syncthreads();
        hr[k * 16 + e] = dsub(dscale(x, 0.5), dscale(abdc(sG, sX, sG), 0.5));
    }
}

// Gradient and HVP of C = 1 - (1/N_s) sum |T_s|^2 per gate, then the tangent-space
// projections of App. F. Block k handles gate k with 16 threads (one per entry).
__global__ void grad_kernel(const double* __restrict__ env, const double2* __restrict__ G,
                            const double2* __restrict__ V, const double2* __restrict__ T,
                            const double2* __restrict__ Om, double2* ge, double2* he, double2* gr, double2* hr,
                            int K, int ns, int tangent, int frob) {
    const int k = blockIdx.x, e = threadIdx.x;
    double2 g = make_double2(0.0, 0.0), h = make_double2(0.0, 0.0);
    for (int s = 0; s < ns; ++s) {
        const double2* Es = reinterpret_cast<const double2*>(env + ((size_t)s * K + k) * 64);
        const double2 E = dconj(Es[e]);
        if (frob) {                                     // C_F: -(1/N) sum conj(E_s), conj(DE_s)
            g = dadd(g, E);
            if (tangent) h = dadd(h, dconj(Es[16 + e]));
        } else {
            g = dadd(g, dmul(T[s], E));                 // T_s conj(E_s)
            if (tangent) {
                h = dadd(h, dmul(Om[s], E));            // Omega_s conj(E_s)
                h = dadd(h, dmul(T[s], dconj(Es[16 + e])));  // T_s conj(DE_s)
            }
        }
    }
    const double scale = (frob ? -1.0 : -2.0) / ns;
    finish_gate(k, e, dscale(g, scale), dscale(h, scale), G, V, ge, he, gr, hr, tangent);
}

// The same from sample-summed weighted environments (the fused-block
// schedule): Ew = sum_s conj(T_s) E_s and DEw = sum_s (conj(Omega_s) E_s +
// conj(T_s) DE_s) (with weights 1 and 0 for the Frobenius cost), so
// grad = scale conj(Ew) and H[V] = scale conj(DEw).
__global__ void weighted_grad_kernel(const double2* __restrict__ Ew, const double2* __restrict__ DEw,
                                     const double2* __restrict__ G, const double2* __restrict__ V, double2* ge,
                                     double2* he, double2* gr, double2* hr, int K, double scale, int tangent) {
    const int k = blockIdx.x, e = threadIdx.x;
    const double2 g = dscale(dconj(Ew[k * 16 + e]), scale);
    const double2 h = tangent ? dscale(dconj(DEw[k * 16 + e]), scale) : make_double2(0.0, 0.0);
    finish_gate(k, e, g, h, G, V, ge, he, gr, hr, tangent);
}

__global__ void loss_kernel(const double2* __restrict__ T, double* loss, int ns, int frob) {
    __shared__ double sh[256];
    double a = 0.0;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) a += frob ? T[s].x : T[s].x * T[s].x + T[s].y * T[s].y;
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss[0] = 1.0 - sh[0] / ns;   // Eq. costHS (Eq. Frobenius with frob)
}

__global__ void psi1q_convert_kernel(const double* __restrict__ in, float2* out, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = make_float2((float)in[2 * i], (float)in[2 * i + 1]);
}

// Standard layout (qubit q on bit n-1-q) -> plan layout (qubit q on bit pos[q]).
__global__ void phi_permute_kernel(const double2* __restrict__ in, void* out, int dbl, int n, int ns,
                                   const int* __restrict__ pos) {
    const size_t dim = (size_t)1 << n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < dim * ns; i += (size_t)gridDim.x * blockDim.x) {
        const size_t s = i >> n, x = i & (dim - 1);
        size_t y = 0;
        for (int q = 0; q < n; ++q) y |= ((x >> (n - 1 - q)) & 1) << pos[q];
        const double2 v = in[i];
        if (dbl) reinterpret_cast<double2*>(out)[s * dim + y] = v;
        else reinterpret_cast<float2*>(out)[s * dim + y] = make_float2((float)v.x, (float)v.y);
    }
}

// Translation-invariant layers (App. E): every gate of layer l is the layer
// gate G_l (and the direction V_l). One CTA of 16 threads per layer.
__global__ void expand_layers_kernel(const double2* __restrict__ GL, const double2* __restrict__ VL,
                                     double2* __restrict__ G, double2* __restrict__ V,
                                     const int* __restrict__ first) {
    const int l = blockIdx.x, e = threadIdx.x;
    const double2 g = GL[l * 16 + e];
    const double2 v = VL ? VL[l * 16 + e] : make_double2(0.0, 0.0);
    for (int k = first[l]; k < first[l + 1]; ++k) {
        G[k * 16 + e] = g;
        if (VL) V[k * 16 + e] = v;
    }
}

// The chain rule through the tying map of App. E: the derivative with respect
// to a layer gate is the sum of the per-gate blocks of its layer (gradient
// and HVP alike; the Riemannian forms are linear in those blocks at a fixed
// layer gate, so they sum the same way). FP64, gates in circuit order. Grid
// (layer, output): outputs 0..3 = Euclidean gradient, Euclidean HVP,
// Riemannian gradient, Riemannian HVP, each K x 16 per gate in `in` and
// n_layers x 16 per layer in `out`.
__global__ void contract_layers_kernel(const double2* __restrict__ in, double2* __restrict__ out,
                                       const int* __restrict__ first, int L, int K) {
    const int l = blockIdx.x, which = blockIdx.y, e = threadIdx.x;
    const double2* src = in + (size_t)which * K * 16;
    double2 a = make_double2(0.0, 0.0);
    for (int k = first[l]; k < first[l + 1]; ++k) a = dadd(a, src[k * 16 + e]);
    out[((size_t)which * L + l) * 16 + e] = a;
}

}  // namespace

cudaError_t launch_expand_layers(const double2* GL, const double2* VL, double2* G, double2* V, const int* first, int L,
                                 cudaStream_t st) {
    expand_layers_kernel<<<L, 16, 0, st>>>(GL, VL, G, V, first);
    return cudaGetLastError();
}

cudaError_t launch_contract_layers(const double2* per_gate, double2* per_layer, const int* first, int L, int K,
                                   cudaStream_t st) {
    contract_layers_kernel<<<dim3(L, 4), 16, 0, st>>>(per_gate, per_layer, first, L, K);
    return cudaGetLastError();
}

cudaError_t launch_prep(const double2* G, const double2* V, void* mats, bool dbl, int K, int* status,
                        cudaStream_t st) {
    prep_kernel<<<(K + 63) / 64, 64, 0, st>>>(G, V, mats, dbl ? 1 : 0, K, status);
    return cudaGetLastError();
}

cudaError_t launch_post(const PostArgs& p, cudaStream_t st) {
    const int pairs = p.K * p.n_samples;
    reduce_kernel<<<(pairs + 7) / 8, 256, 0, st>>>(p.partial, p.env, p.K, p.n_samples, p.cx_count);
    overlaps_kernel<<<p.n_samples, 256, 0, st>>>(p.env, p.G, p.V, p.T, p.Omega, p.K, p.tangent);
    grad_kernel<<<p.K, 16, 0, st>>>(p.env, p.G, p.V, p.T, p.Omega, p.grad_e, p.hvp_e, p.grad_r, p.hvp_r, p.K,
                                     p.n_samples, p.tangent, p.frobenius);
    loss_kernel<<<1, 256, 0, st>>>(p.T, p.loss, p.n_samples, p.frobenius);
    return cudaGetLastError();
}

cudaError_t launch_post_weighted(const double2* Ew, const double2* DEw, const double2* G, const double2* V,
                                 const double2* T, double2* ge, double2* he, double2* gr, double2* hr, double* loss,
                                 int K, int ns, int tangent, int frob, cudaStream_t st) {
    const double scale = (frob ? -1.0 : -2.0) / ns;
    weighted_grad_kernel<<<K, 16, 0, st>>>(Ew, DEw, G, V, ge, he, gr, hr, K, scale, tangent);
    loss_kernel<<<1, 256, 0, st>>>(T, loss, ns, frob);
    return cudaGetLastError();
}

cudaError_t launch_psi1q_convert(const double* in, float2* out, size_t count, cudaStream_t st) {
    psi1q_convert_kernel<<<(int)((count + 255) / 256), 256, 0, st>>>(in, out, count);
    return cudaGetLastError();
}

cudaError_t launch_phi_permute(const double2* phi_std, void* phi_out, bool dbl, int n, int ns, const int* pos,
                               cudaStream_t st) {
    const size_t total = ((size_t)1 << n) * ns;
    size_t blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    phi_permute_kernel<<<(int)blocks, 256, 0, st>>>(phi_std, phi_out, dbl ? 1 : 0, n, ns, pos);
    return cudaGetLastError();
}

}  // namespace hvp
