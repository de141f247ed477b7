/*
 * FP64 CPU oracle for the sampled Hilbert-Schmidt loss of a brickwall
 * circuit, its complex gradient and its Hessian-vector product.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. It shares no code,
 * header, table or helper with the CUDA library; both sides only consume the
 * same seeded inputs.
 *
 * What it computes (arXiv 2604.20384):
 *   - states:    psi^[k] = G_k psi^[k-1]                         (Eq. fis)
 *                phi^[k] = G_{K-k+1}^dagger phi^[k-1]           (Eq. bis)
 *   - tangents:  dpsi^[k] = G_k dpsi^[k-1] + V_k psi^[k-1]        (Eq. dfis)
 *                dphi^[k] = G_{K-k+1}^dag dphi^[k-1]
 *                           + V_{K-k+1}^dag phi^[k-1]             (Eq. dbis)
 *   - environment of gate k:
 *                E_k[i][j]  = sum_a conj(phi^[K-k]_{i a}) psi^[k-1]_{j a}
 *                                                       (Eq. environment)
 *                DE_k[i][j] = sum_a conj(dphi^[K-k]_{i a}) psi^[k-1]_{j a}
 *                           + sum_a conj(phi^[K-k]_{i a}) dpsi^[k-1]_{j a}
 *                                                       (Eq. Dpsi / overlap-hvp)
 *   - overlap T = phi^dagger G psi, taken at the boundary (Alg. 1);
 *     Omega = sum_k sum_ij E_k[i][j] V_k[i][j]           (Eq. Omega, App. B)
 *   - loss  C = 1 - (1/N_s) sum_s |T_s|^2                 (Eq. costHS)
 *   - gradient and HVP of C (Alg. 2 post-processing, Eq. grad-costHS,
 *     Eq. hvp-costHS), Riemannian forms (App. F, Eq. projec).
 *   - the Frobenius cost C_F = 1 - (1/N_s) sum_s Re T_s (Eq. Frobenius), its
 *     gradient -(1/N_s) sum_s conj(E_s) (Eq. grad-costF) and HVP
 *     -(1/N_s) sum_s conj(DE_s) (Eq. hvp-costF), with Riemannian forms.
 *
 * Readings of the paper taken here:
 *   (1) Alg. 1 updates dphi before it is used in the HVP line; Eq. overlap-hvp
 *       needs the value before the update. This oracle uses phi^[K-k] and
 *       dphi^[K-k] (pre-update) for gate k, then updates dphi, then phi.
 *   (2) Eq. grad-costHS is the gradient of +|T|^2 and Eq. hvp-costHS the HVP
 *       of -|T|^2. All outputs here are derivatives of the sampled cost C of
 *       Eq. costHS: grad C = -(1/N_s) sum_s 2 T_s conj(E_s) and
 *       H C[V] = -(1/N_s) sum_s 2 (Omega_s conj(E_s) + T_s conj(DE_s)),
 *       i.e. the forward-over-reverse definition (Eq. FoR) applied to C.
 *   (3) Eq. costHS is missing a dagger; it reads |phi_s^dagger G psi_s|^2.
 *   (4) The complex gradient of a real f is df/dx + i df/dy (Eq. grad-real).
 *
 * Conventions (the paper is silent): qubit 0 is the most significant bit of
 * an amplitude index; layer l (1-based) has offset (l-1) mod 2 and gates on
 * (i, i+1), i = offset, offset+2, ..., i+1 <= n-1; gates are ordered
 * layer-major then by i; a gate's 4x4 matrix is indexed by 2 b_i + b_{i+1}
 * and stored row-major as interleaved (re, im) doubles.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* Brickwall layout (Sec. 3.1, Fig. computational-passes).             */
/* ------------------------------------------------------------------ */

/* Fills first_qubit[k] (may be NULL) and returns K. */
int oracle_layout(int n, int n_layers, int *first_qubit)
{
    int k = 0;
    for (int layer = 1; layer <= n_layers; ++layer) {
        int offset = (layer - 1) % 2;
        for (int i = offset; i + 1 <= n - 1; i += 2) {
            if (first_qubit) first_qubit[k] = i;
            ++k;
        }
    }
    return k;
}

/* ------------------------------------------------------------------ */
/* Small dense helpers on 4x4 complex matrices.                        */
/* ------------------------------------------------------------------ */

static void load4(const double *src, cplx *m)
{
    for (int e = 0; e < 16; ++e) m[e] = src[2 * e] + I * src[2 * e + 1];
}

static void store4(const cplx *m, double *dst)
{
    for (int e = 0; e < 16; ++e) { dst[2 * e] = creal(m[e]); dst[2 * e + 1] = cimag(m[e]); }
}

static void adjoint4(const cplx *m, cplx *out)
{
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) out[r * 4 + c] = conj(m[c * 4 + r]);
}

static void matmul4(const cplx *a, const cplx *b, cplx *out)
{
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            cplx acc = 0;
            for (int t = 0; t < 4; ++t) acc += a[r * 4 + t] * b[t * 4 + c];
            out[r * 4 + c] = acc;
        }
}

/* Tangent-space projection P_G(X) = X/2 - G X^dagger G / 2 (App. F, Eq. projec). */
static void project4(const cplx *g, const cplx *x, cplx *out)
{
    cplx xd[16], t[16], gxdg[16];
    adjoint4(x, xd);
    matmul4(g, xd, t);
    matmul4(t, g, gxdg);
    for (int e = 0; e < 16; ++e) out[e] = 0.5 * x[e] - 0.5 * gxdg[e];
}

/* ------------------------------------------------------------------ */
/* State-vector operations.                                            */
/* ------------------------------------------------------------------ */

/* Amplitude offsets of the four basis states 2 b_q + b_{q+1} of a gate on
 * qubits (q, q+1), for a base index x with both bits clear. */
static void gate_offsets(int n, int q, size_t *sh, size_t *sl)
{
    *sh = (size_t)1 << (n - 1 - q);  /* qubit q      */
    *sl = (size_t)1 << (n - 2 - q);  /* qubit q + 1  */
}

/* psi <- M psi on qubits (q, q+1). */
static void apply_gate(cplx *psi, int n, int q, const cplx *m)
{
    size_t sh, sl, dim = (size_t)1 << n;
    gate_offsets(n, q, &sh, &sl);
    for (size_t x = 0; x < dim; ++x) {
        if (x & (sh | sl)) continue;
        size_t idx[4] = {x, x | sl, x | sh, x | sh | sl};
        cplx in[4], out[4];
        for (int c = 0; c < 4; ++c) in[c] = psi[idx[c]];
        for (int r = 0; r < 4; ++r) {
            out[r] = 0;
            for (int c = 0; c < 4; ++c) out[r] += m[r * 4 + c] * in[c];
        }
        for (int r = 0; r < 4; ++r) psi[idx[r]] = out[r];
    }
}

/* (psi, dpsi) <- (M psi, M dpsi + W psi) on qubits (q, q+1): one step of
 * Eq. fis together with Eq. dfis (or, with adjoints, Eq. bis with Eq. dbis). */
static void apply_gate_tangent(cplx *psi, cplx *dpsi, int n, int q,
                               const cplx *m, const cplx *w)
{
    size_t sh, sl, dim = (size_t)1 << n;
    gate_offsets(n, q, &sh, &sl);
    for (size_t x = 0; x < dim; ++x) {
        if (x & (sh | sl)) continue;
        size_t idx[4] = {x, x | sl, x | sh, x | sh | sl};
        cplx p[4], d[4], po[4], dout[4];
        for (int c = 0; c < 4; ++c) { p[c] = psi[idx[c]]; d[c] = dpsi[idx[c]]; }
        for (int r = 0; r < 4; ++r) {
            po[r] = 0; dout[r] = 0;
            for (int c = 0; c < 4; ++c) {
                po[r] += m[r * 4 + c] * p[c];
                dout[r] += m[r * 4 + c] * d[c] + w[r * 4 + c] * p[c];
            }
        }
        for (int r = 0; r < 4; ++r) { psi[idx[r]] = po[r]; dpsi[idx[r]] = dout[r]; }
    }
}

/* acc[i][j] += sum_a conj(x_{i a}) y_{j a} over the other qubits
 * (the partial contraction of Eq. environment). */
static void env_accumulate(const cplx *x, const cplx *y, int n, int q, cplx *acc)
{
    size_t sh, sl, dim = (size_t)1 << n;
    gate_offsets(n, q, &sh, &sl);
    for (size_t base = 0; base < dim; ++base) {
        if (base & (sh | sl)) continue;
        size_t idx[4] = {base, base | sl, base | sh, base | sh | sl};
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) acc[i * 4 + j] += conj(x[idx[i]]) * y[idx[j]];
    }
}

static cplx inner(const cplx *x, const cplx *y, size_t dim)  /* x^dagger y */
{
    cplx acc = 0;
    for (size_t e = 0; e < dim; ++e) acc += conj(x[e]) * y[e];
    return acc;
}

/* psi_s = tensor product of the n single-qubit states (Eq. costHS: Haar
 * product states); qubit 0 is the most significant bit. */
static void product_state(const double *psi1q_s, int n, cplx *psi)
{
    size_t dim = (size_t)1 << n;
    for (size_t x = 0; x < dim; ++x) {
        cplx amp = 1;
        for (int q = 0; q < n; ++q) {
            int bit = (int)((x >> (n - 1 - q)) & 1);
            amp *= psi1q_s[4 * q + 2 * bit] + I * psi1q_s[4 * q + 2 * bit + 1];
        }
        psi[x] = amp;
    }
}

/* ------------------------------------------------------------------ */
/* Reference states phi_s = U_ref psi_s (Sec. 3.1: phi = U_ref psi).   */
/* ------------------------------------------------------------------ */

int oracle_reference_states(int n, int n_layers, int n_samples, const double *uref,
                            const double *psi1q, double *phi_out)
{
    int K = oracle_layout(n, n_layers, NULL);
    int *fq = malloc(sizeof(int) * (K > 0 ? K : 1));
    size_t dim = (size_t)1 << n;
    cplx *psi = malloc(sizeof(cplx) * dim);
    if (!fq || !psi) { free(fq); free(psi); return -2; }
    oracle_layout(n, n_layers, fq);
    for (int s = 0; s < n_samples; ++s) {
        product_state(psi1q + (size_t)s * n * 4, n, psi);
        for (int k = 0; k < K; ++k) {
            cplx u[16];
            load4(uref + (size_t)k * 32, u);
            apply_gate(psi, n, fq[k], u);
        }
        for (size_t x = 0; x < dim; ++x) {
            phi_out[((size_t)s * dim + x) * 2] = creal(psi[x]);
            phi_out[((size_t)s * dim + x) * 2 + 1] = cimag(psi[x]);
        }
    }
    free(fq); free(psi);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Alg. 1 for one sample.                                              */
/* ------------------------------------------------------------------ */

typedef struct {
    int n, K, with_tangent, ckpt_stride;
    const int *fq;
    const cplx *G, *Gd, *V, *Vd;   /* K x 16 each; Vd = V^dagger       */
    const double *psi1q;            /* N_s x n x 2 complex              */
    const double *phi;              /* N_s x 2^n complex                */
    /* per-sample outputs */
    cplx *T, *Omega, *Omega_fwd;    /* N_s                              */
    cplx *E, *DE;                   /* N_s x K x 16                     */
    cplx *cuts;                     /* N_s x (K+1), may be NULL         */
    int n_samples, n_threads;
    int error;
} job_t;

typedef struct { job_t *job; int tid; } worker_arg_t;

/* Runs the forward pass (caching psi^[k], dpsi^[k] every ckpt_stride gates)
 * and the backward pass of Alg. 1 for sample s. With ckpt_stride > 1 the
 * states between checkpoints are recomputed from the nearest checkpoint,
 * segment by segment, which gives the same states as a full cache. */
static int run_sample(const job_t *jb, int s, cplx *work)
{
    const int n = jb->n, K = jb->K, c = jb->ckpt_stride, tan = jb->with_tangent;
    const size_t dim = (size_t)1 << n;
    const int n_ckpt = K / c + 1;                 /* checkpoints at k = 0, c, 2c, ... */
    cplx *ck_psi = work;                          /* n_ckpt x dim */
    cplx *ck_dpsi = ck_psi + (size_t)n_ckpt * dim;
    cplx *seg_psi = ck_dpsi + (size_t)n_ckpt * dim;   /* c x dim */
    cplx *seg_dpsi = seg_psi + (size_t)c * dim;
    cplx *phi = seg_dpsi + (size_t)c * dim;
    cplx *dphi = phi + dim;
    cplx *cur = dphi + dim, *dcur = cur + dim;

    /* Forward pass (Alg. 1, first procedure): psi^[0] = product state,
     * dpsi^[0] = 0. */
    product_state(jb->psi1q + (size_t)s * n * 4, n, cur);
    memset(dcur, 0, sizeof(cplx) * dim);
    for (int k = 0; k <= K; ++k) {
        if (k % c == 0) {
            memcpy(ck_psi + (size_t)(k / c) * dim, cur, sizeof(cplx) * dim);
            memcpy(ck_dpsi + (size_t)(k / c) * dim, dcur, sizeof(cplx) * dim);
        }
        if (k == K) break;
        if (tan) apply_gate_tangent(cur, dcur, n, jb->fq[k], jb->G + 16 * k, jb->V + 16 * k);
        else apply_gate(cur, n, jb->fq[k], jb->G + 16 * k);
    }
    /* cur, dcur now hold psi^[K], dpsi^[K]. */
    for (size_t x = 0; x < dim; ++x)
        phi[x] = jb->phi[((size_t)s * dim + x) * 2] + I * jb->phi[((size_t)s * dim + x) * 2 + 1];
    memset(dphi, 0, sizeof(cplx) * dim);
    if (jb->cuts) jb->cuts[(size_t)s * (K + 1) + K] = inner(phi, cur, dim);
    /* Omega via the forward tangent state: D T[V] = phi^dagger dpsi^[K]. */
    jb->Omega_fwd[s] = tan ? inner(phi, dcur, dim) : 0;

    /* Backward pass (Alg. 1, second procedure), k = K..1 (0-based k-1). */
    int seg_lo = -1;  /* first gate index whose input state is in seg_* */
    for (int k = K; k >= 1; --k) {
        int kk = k - 1;                   /* 0-based gate index */
        /* psi^[k-1], dpsi^[k-1]: from the segment buffer, recomputed from
         * the checkpoint at floor((k-1)/c)*c when needed. */
        int base = ((k - 1) / c) * c;
        if (seg_lo != base) {
            memcpy(cur, ck_psi + (size_t)(base / c) * dim, sizeof(cplx) * dim);
            memcpy(dcur, ck_dpsi + (size_t)(base / c) * dim, sizeof(cplx) * dim);
            for (int j = base; j < base + c && j < K; ++j) {
                memcpy(seg_psi + (size_t)(j - base) * dim, cur, sizeof(cplx) * dim);
                memcpy(seg_dpsi + (size_t)(j - base) * dim, dcur, sizeof(cplx) * dim);
                if (j + 1 < base + c) {
                    if (tan) apply_gate_tangent(cur, dcur, n, jb->fq[j], jb->G + 16 * j, jb->V + 16 * j);
                    else apply_gate(cur, n, jb->fq[j], jb->G + 16 * j);
                }
            }
            seg_lo = base;
        }
        const cplx *psi_km1 = seg_psi + (size_t)(k - 1 - base) * dim;
        const cplx *dpsi_km1 = seg_dpsi + (size_t)(k - 1 - base) * dim;

        /* Gradient and HVP blocks with the pre-update phi^[K-k], dphi^[K-k]
         * (reading (1)). */
        cplx *Ek = jb->E + ((size_t)s * K + kk) * 16;
        cplx *DEk = jb->DE + ((size_t)s * K + kk) * 16;
        memset(Ek, 0, sizeof(cplx) * 16);
        memset(DEk, 0, sizeof(cplx) * 16);
        env_accumulate(phi, psi_km1, n, jb->fq[kk], Ek);
        if (tan) {
            env_accumulate(dphi, psi_km1, n, jb->fq[kk], DEk);
            env_accumulate(phi, dpsi_km1, n, jb->fq[kk], DEk);
        }
        /* Then dphi <- G^dag dphi + V^dag phi, phi <- G^dag phi (Eq. dbis, bis). */
        if (tan) apply_gate_tangent(phi, dphi, n, jb->fq[kk], jb->Gd + 16 * kk, jb->Vd + 16 * kk);
        else apply_gate(phi, n, jb->fq[kk], jb->Gd + 16 * kk);
        if (jb->cuts) jb->cuts[(size_t)s * (K + 1) + (k - 1)] = inner(phi, psi_km1, dim);
    }
    /* T at the boundary: T = phi^[K]^dagger psi^[0] (Alg. 1, last line). */
    memcpy(cur, ck_psi, sizeof(cplx) * dim);
    jb->T[s] = inner(phi, cur, dim);
    /* Omega = sum_k sum_ij (dT/dG_k)_ij V_k,ij (Eq. Omega, App. B). */
    cplx om = 0;
    if (tan)
        for (int kk = 0; kk < K; ++kk)
            for (int e = 0; e < 16; ++e) om += jb->E[((size_t)s * K + kk) * 16 + e] * jb->V[16 * kk + e];
    jb->Omega[s] = om;
    return 0;
}

static void *worker(void *p)
{
    worker_arg_t *wa = p;
    job_t *jb = wa->job;
    const size_t dim = (size_t)1 << jb->n;
    const int c = jb->ckpt_stride;
    const size_t n_states = 2 * (size_t)(jb->K / c + 1) + 2 * (size_t)c + 4;
    cplx *work = malloc(sizeof(cplx) * dim * n_states);
    if (!work) { jb->error = -2; return NULL; }
    for (int s = wa->tid; s < jb->n_samples; s += jb->n_threads) run_sample(jb, s, work);
    free(work);
    return NULL;
}

/*
 * Full evaluation. Arrays are interleaved complex128 (re, im):
 *   G, V: K x 4 x 4 (V may be NULL: loss and gradient only)
 *   psi1q: N_s x n x 2; phi: N_s x 2^n (the reference states U_ref psi_s)
 * Outputs (any may be NULL):
 *   loss[1]; T, Omega, Omega_fwd: N_s; E, DE: N_s x K x 16; grad, hvp,
 *   grad_r, hvp_r: K x 16; cuts: N_s x (K+1) overlaps phi^[K-k]^dag psi^[k].
 * ckpt_stride >= 1: checkpoint spacing of the forward cache (1 = every gate).
 * Returns 0, -1 on bad arguments, -2 on allocation failure.
 */
int oracle_hvp(int n, int n_layers, int n_samples,
               const double *G_in, const double *V_in, const double *psi1q, const double *phi,
               int ckpt_stride, int n_threads,
               double *loss, double *T_out, double *Omega_out, double *Omega_fwd_out,
               double *E_out, double *DE_out,
               double *grad, double *hvp, double *grad_r, double *hvp_r, double *cuts_out,
               double *loss_f, double *grad_f, double *hvp_f, double *grad_fr, double *hvp_fr)
{
    if (n < 2 || n > 30 || n_layers < 1 || n_samples < 1 || ckpt_stride < 1 || !G_in || !psi1q || !phi)
        return -1;
    int K = oracle_layout(n, n_layers, NULL);
    int tan = V_in != NULL;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_samples) n_threads = n_samples;

    int *fq = malloc(sizeof(int) * K);
    cplx *G = malloc(sizeof(cplx) * 16 * K), *Gd = malloc(sizeof(cplx) * 16 * K);
    cplx *V = calloc((size_t)16 * K, sizeof(cplx)), *Vd = calloc((size_t)16 * K, sizeof(cplx));
    cplx *T = malloc(sizeof(cplx) * n_samples), *Om = malloc(sizeof(cplx) * n_samples);
    cplx *Omf = malloc(sizeof(cplx) * n_samples);
    cplx *E = malloc(sizeof(cplx) * 16 * (size_t)K * n_samples);
    cplx *DE = malloc(sizeof(cplx) * 16 * (size_t)K * n_samples);
    cplx *cuts = cuts_out ? malloc(sizeof(cplx) * (size_t)(K + 1) * n_samples) : NULL;
    pthread_t *th = malloc(sizeof(pthread_t) * n_threads);
    worker_arg_t *wa = malloc(sizeof(worker_arg_t) * n_threads);
    int rc = 0;
    if (!fq || !G || !Gd || !V || !Vd || !T || !Om || !Omf || !E || !DE || !th || !wa ||
        (cuts_out && !cuts)) { rc = -2; goto done; }

    oracle_layout(n, n_layers, fq);
    for (int k = 0; k < K; ++k) {
        load4(G_in + 32 * (size_t)k, G + 16 * k);
        adjoint4(G + 16 * k, Gd + 16 * k);
        if (tan) { load4(V_in + 32 * (size_t)k, V + 16 * k); adjoint4(V + 16 * k, Vd + 16 * k); }
    }

    job_t jb = {n, K, tan, ckpt_stride, fq, G, Gd, V, Vd, psi1q, phi,
                T, Om, Omf, E, DE, cuts, n_samples, n_threads, 0};
    for (int t = 0; t < n_threads; ++t) {
        wa[t].job = &jb; wa[t].tid = t;
        if (pthread_create(&th[t], NULL, worker, &wa[t]) != 0) { n_threads = t; jb.error = -2; break; }
    }
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    if (jb.error) { rc = jb.error; goto done; }

    /* Alg. 2 post-processing in sample order (deterministic). */
    const double inv_n = 1.0 / n_samples;
    double fid = 0;
    for (int s = 0; s < n_samples; ++s) fid += creal(T[s] * conj(T[s]));
    if (loss) loss[0] = 1.0 - inv_n * fid;              /* Eq. costHS */
    double reT = 0;
    for (int s = 0; s < n_samples; ++s) reT += creal(T[s]);
    if (loss_f) loss_f[0] = 1.0 - inv_n * reT;          /* Eq. Frobenius, sampled */

    for (int k = 0; k < K; ++k) {
        cplx g[16] = {0}, h[16] = {0};
        for (int s = 0; s < n_samples; ++s) {
            const cplx *Es = E + ((size_t)s * K + k) * 16, *DEs = DE + ((size_t)s * K + k) * 16;
            for (int e = 0; e < 16; ++e) {
                cplx gradF = -conj(Es[e]);                  /* grad L_F = -conj(dT/dG) (Eq. grad-costF) */
                cplx grad_abs2 = -2.0 * T[s] * gradF;      /* grad |T|^2 (Eq. grad-costHS) */
                g[e] += -inv_n * grad_abs2;                 /* grad of 1 - mean |T|^2 */
                if (tan) {
                    cplx hvpF = -conj(DEs[e]);              /* H L_F[V] (Eq. hvp-costF) */
                    /* D(grad |T|^2)[V] = -2 (Omega grad L_F + T H L_F[V]), the product
                     * rule of App. A applied to -2 T grad L_F (reading (2)). */
                    cplx hvp_abs2 = -2.0 * (Om[s] * gradF + T[s] * hvpF);
                    h[e] += -inv_n * hvp_abs2;
                }
            }
        }
        if (grad) store4(g, grad + 32 * (size_t)k);
        if (hvp) store4(h, hvp + 32 * (size_t)k);
        /* Frobenius cost: grad L_F = -conj(dT/dG) (Eq. grad-costF),
         * H L_F[V] = -conj(D(dT/dG)[V]) (Eq. hvp-costF), averaged over samples. */
        cplx gf[16] = {0}, hf[16] = {0};
        for (int s = 0; s < n_samples; ++s)
            for (int e = 0; e < 16; ++e) {
                gf[e] += -inv_n * conj(E[((size_t)s * K + k) * 16 + e]);
                if (tan) hf[e] += -inv_n * conj(DE[((size_t)s * K + k) * 16 + e]);
            }
        if (grad_f) store4(gf, grad_f + 32 * (size_t)k);
        if (hvp_f) store4(hf, hvp_f + 32 * (size_t)k);
        if (grad_fr || hvp_fr) {
            const cplx *Gk = G + 16 * k, *Vk = V + 16 * k;
            cplx pr[16], gd[16], t1[16], t2[16], t3[16], t4[16], x[16];
            project4(Gk, gf, pr);
            if (grad_fr) store4(pr, grad_fr + 32 * (size_t)k);
            if (hvp_fr) {
                adjoint4(gf, gd);
                matmul4(Vk, gd, t1); matmul4(t1, Gk, t2);
                matmul4(Gk, gd, t3); matmul4(t3, Vk, t4);
                for (int e = 0; e < 16; ++e) x[e] = hf[e] - 0.5 * t2[e] - 0.5 * t4[e];
                project4(Gk, x, pr);
                store4(pr, hvp_fr + 32 * (size_t)k);
            }
        }
        if (grad_r || hvp_r) {
            /* App. F: grad_R = P_G(grad);
             * H_R[V] = P_G(H[V] - V grad^dag G / 2 - G grad^dag V / 2). */
            const cplx *Gk = G + 16 * k, *Vk = V + 16 * k;
            cplx gr[16], gd[16], t1[16], t2[16], t3[16], t4[16], x[16], hr[16];
            project4(Gk, g, gr);
            if (grad_r) store4(gr, grad_r + 32 * (size_t)k);
            if (hvp_r) {
                adjoint4(g, gd);
                matmul4(Vk, gd, t1); matmul4(t1, Gk, t2);   /* V grad^dag G */
                matmul4(Gk, gd, t3); matmul4(t3, Vk, t4);   /* G grad^dag V */
                for (int e = 0; e < 16; ++e) x[e] = h[e] - 0.5 * t2[e] - 0.5 * t4[e];
                project4(Gk, x, hr);
                store4(hr, hvp_r + 32 * (size_t)k);
            }
        }
    }
    for (int s = 0; s < n_samples; ++s) {
        if (T_out) { T_out[2 * s] = creal(T[s]); T_out[2 * s + 1] = cimag(T[s]); }
        if (Omega_out) { Omega_out[2 * s] = creal(Om[s]); Omega_out[2 * s + 1] = cimag(Om[s]); }
        if (Omega_fwd_out) { Omega_fwd_out[2 * s] = creal(Omf[s]); Omega_fwd_out[2 * s + 1] = cimag(Omf[s]); }
    }
    if (E_out)
        for (size_t e = 0; e < 16 * (size_t)K * n_samples; ++e) { E_out[2 * e] = creal(E[e]); E_out[2 * e + 1] = cimag(E[e]); }
    if (DE_out)
        for (size_t e = 0; e < 16 * (size_t)K * n_samples; ++e) { DE_out[2 * e] = creal(DE[e]); DE_out[2 * e + 1] = cimag(DE[e]); }
    if (cuts_out)
        for (size_t e = 0; e < (size_t)(K + 1) * n_samples; ++e) { cuts_out[2 * e] = creal(cuts[e]); cuts_out[2 * e + 1] = cimag(cuts[e]); }

done:
    free(fq); free(G); free(Gd); free(V); free(Vd); free(T); free(Om); free(Omf);
    free(E); free(DE); free(cuts); free(th); free(wa);
    return rc;
}

/* P_G(X) for K gates, exposed for the projection pins (App. F, Eq. projec). */
int oracle_project(int K, const double *G_in, const double *X_in, double *out)
{
    for (int k = 0; k < K; ++k) {
        cplx g[16], x[16], p[16];
        load4(G_in + 32 * (size_t)k, g);
        load4(X_in + 32 * (size_t)k, x);
        project4(g, x, p);
        store4(p, out + 32 * (size_t)k);
    }
    return 0;
}
