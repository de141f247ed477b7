/*
 * hvp.h - C ABI of the GB300 (sm_103a) library for the sampled
 * Hilbert-Schmidt loss of a brickwall circuit, its complex gradient and its
 * Hessian-vector product by recursive tangent-state propagation
 * (arXiv 2604.20384).
 *
 * Problem (Sec. 3.1, Eq. HST; Sec. 4.1, Eq. costHS; Alg. 2 "Require" line):
 * given a brickwall of K two-qubit gates G = (G^[1], ..., G^[K]) on n qubits,
 * N_s product input states psi_s and reference states phi_s = U_ref psi_s,
 *     C(G) = 1 - (1/N_s) sum_s |phi_s^dagger G_K ... G_1 psi_s|^2 .
 * The library returns C, the complex gradient grad C (Eq. grad-real:
 * dC/dRe + i dC/dIm per matrix entry) and the HVP H C[V] = D(grad C)[V]
 * along a direction V (Eq. FoR), optionally projected to the tangent space
 * of U(4)^K (App. F, Eq. projec).
 *
 * Conventions for every array (the paper is silent on them):
 *   - complex numbers are interleaved (re, im) doubles;
 *   - qubit 0 is the most significant bit of an amplitude index;
 *   - layer l (1-based) has offset (l-1) mod 2 and gates on qubits (i, i+1),
 *     i = offset, offset+2, ..., i+1 <= n-1; gates are numbered layer-major,
 *     then by i; K = hvp_num_gates(n, n_layers);
 *   - a gate is a 4x4 row-major matrix indexed by 2 b_i + b_{i+1};
 *     G, V, grad and hvp arrays hold K*16 complex numbers = K*32 doubles;
 *   - psi_1q holds N_s*n single-qubit states (2 complex each) = N_s*n*4
 *     doubles, psi_s = psi_{s,0} (x) ... (x) psi_{s,n-1};
 *   - a state vector holds 2^n complex numbers.
 *
 * Ownership: the caller owns every array it passes. The library copies
 * inputs and never keeps a caller pointer after a call returns. A context
 * owns all device memory it allocates; hvp_free releases it.
 *
 * Errors: every int-returning call returns HVP_OK (0) or a negative code;
 * hvp_last_error gives a message. Calls on one context must not overlap;
 * distinct contexts are independent. A failed hvp_init / hvp_init_batch
 * releases everything it allocated. For tests of that path, the environment
 * variable HVP_DEVICE_ALLOC_CAP_MB caps the device memory one context (or
 * batch) may allocate: an allocation beyond it fails with HVP_ENOMEM as if
 * cudaMalloc had failed.
 *
 * Gates are not required to be unitary (finite differences evaluate G + hV);
 * they must be invertible, because the backward sweep recomputes earlier
 * forward states with G^-1 inside each window pass. The Riemannian outputs
 * assume unitary gates.
 */
#ifndef HVP_H
#define HVP_H

#ifdef __cplusplus
extern "C" {
#endif

#define HVP_OK 0
#define HVP_EINVAL (-1)      /* bad shape, flag, size or NULL pointer          */
#define HVP_ENOMEM (-2)      /* device or host allocation failed               */
#define HVP_ECUDA (-3)       /* a CUDA runtime call or kernel launch failed    */
#define HVP_ETIMEOUT (-4)    /* a bounded device-side wait expired             */
#define HVP_ENONFINITE (-5)  /* NaN/Inf in the inputs or a singular gate       */

/* precision */
#define HVP_C64 0   /* complex64 state sweeps, FP64 per-gate accumulation   */
#define HVP_C128 1  /* complex128 sweeps and FP64 accumulation             */

/* flags */
#define HVP_RIEMANNIAN 1  /* grad/hvp outputs are the Riemannian forms (App. F) */
#define HVP_PHI_GIVEN 2   /* ref_data holds phi_s (N_s x 2^n) instead of U_ref */
#define HVP_UNFUSED 4     /* one kernel launch per gate (the plain schedule)    */
#define HVP_NO_GRAPH 8    /* launch kernels directly instead of a CUDA graph
                             (each pass is then also an NVTX range, named
                             with its index; every call is one)            */
#define HVP_AUTOTUNE 16   /* time the window/threads/arithmetic candidates and
                             the fused-block tensor-core schedule at hvp_init
                             and keep the fastest (see hvp_plan_info)        */
#define HVP_FROBENIUS 32  /* loss, gradient and HVP of the sampled Frobenius
                             cost C_F = 1 - (1/N_s) sum_s Re T_s (Eq. Frobenius,
                             Eq. grad-costF, Eq. hvp-costF) instead of C      */
#define HVP_RECOMPUTE 64  /* recompute the forward states inside each window
                             pass with G^-1 instead of keeping the states
                             before every gate in device memory (see
                             checkpoint_stride below)                         */
#define HVP_MULTI_DIR 128 /* size the forward cache for two tangent
                             directions (24 bytes per amplitude per gate), so
                             that hvp_hvp_multi evaluates directions in pairs
                             sharing one sweep; windows of at most 11 qubits */
#define HVP_TENSOR 256    /* fused-block schedule on the tensor cores: the gates
                             are grouped into blocks of 5 neighbouring qubits
                             (App. D's block operator B and its tangent dB),
                             each block applied to all states as the real
                             GEMM [B ; dB] [psi | dpsi] (128 x 64 x 64 per
                             tile of 32 columns) on exact-integer bf16 slices
                             of both operands (tcgen05, sm_103a), the block
                             environments as a TF32 GEMM, the forward states
                             at every block boundary kept in device memory
                             ((blocks + 1) * 16 * 2^n * N_s bytes), the
                             co-states weighted by T_s and Omega_s so that the
                             block environments sum over samples. Needs
                             complex64 and n >= 5; per-sample environments
                             (HVP_OUT_ENV) are not formed                     */
#define HVP_TRANSLATION 512 /* translation-invariant layers (App. E, Alg. 3):
                             every gate of layer l is one layer gate G_l; G and
                             V hold n_layers*32 doubles (one 4x4 block per
                             layer), and grad and hvp (Euclidean and
                             Riemannian) are the derivatives with respect to
                             the layer gates, the sums of the per-gate blocks
                             over each layer, formed in FP64 on the device.
                             Not with HVP_MULTI_DIR; HVP_OUT_ENV stays per gate */

typedef struct hvp_ctx hvp_ctx;

typedef struct {
    int n;                 /* qubits, 2..30                                    */
    int n_layers;          /* brickwall layers L >= 1                          */
    int n_samples;         /* N_s, 1..65535 (2^n * N_s at most 2^34)           */
    int precision;         /* HVP_C64 or HVP_C128                              */
    int flags;             /* HVP_* flags, or-ed                               */
    int checkpoint_stride; /* 0 = automatic: the forward states before every
                              gate are cached, as in Alg. 1, when K state sets
                              (16 * 2^n * N_s bytes each) fit in 85 % of the
                              free device memory and HVP_RECOMPUTE is not set;
                              otherwise forward checkpoints are kept at window-
                              pass boundaries (every pass if memory allows) and
                              the states inside a pass are recomputed with
                              G^-1. c > 0: checkpoints every c passes, the
                              others recomputed (no cache)                     */
    int window;            /* local qubits per shared-memory tile; 0 = auto    */
    int threads;           /* threads per CTA of the window-pass kernels,
                              128 (scalar arithmetic, two CTAs per SM when
                              the tiles fit), 256 or 512; 0 = auto             */
    int variant;           /* arithmetic of the window-pass kernels: 1 scalar
                              FP32 FMA, 2 packed fma.rn.f32x2, 3 scalar with
                              two groups per thread iteration in the backward
                              passes; 0 = auto. The forward-cache schedule
                              runs the scalar kernels: variants 2 and 3 select
                              the recompute schedule                           */
    int device;            /* CUDA device ordinal                              */
    void *stream;          /* cudaStream_t for all work; NULL = own stream     */
} hvp_config;

/* Number of gates K of an open-boundary brickwall (Sec. 3.1); -1 if n < 2
 * or n_layers < 1. No GPU needed. */
int hvp_num_gates(int n, int n_layers);

/* Creates a context: validates cfg, allocates device memory, uploads the
 * input states and computes phi_s = U_ref psi_s once (Sec. 3.1, Eq.
 * cost-summands: phi = U_ref psi) unless HVP_PHI_GIVEN.
 *   psi_1q   : host, N_s*n*4 doubles (see conventions).
 *   ref_data : host, U_ref gates (K*32 doubles), or with HVP_PHI_GIVEN the
 *              reference states phi_s (N_s * 2^n * 2 doubles).
 * On failure *out is NULL; the message is available from hvp_last_error(NULL)
 * on the calling thread. */
int hvp_init(hvp_ctx **out, const hvp_config *cfg, const double *psi_1q,
             const double *ref_data);

/* Batch of independent circuits of uneven size evaluated together (one
 * persistent kernel launch per call). cfgs[c], psi_1q[c] and ref_data[c]
 * describe circuit c exactly as for hvp_init (complex64 path only; flags,
 * device and stream are taken from cfgs[0]). The context then works with the
 * same calls: G, V, grad and hvp concatenate the circuits' gates in order
 * (sum_c K_c * 32 doubles), loss holds one double per circuit, HVP_OUT_T and
 * HVP_OUT_OMEGA concatenate the circuits' samples; HVP_OUT_ENV and
 * hvp_profile are not available. Circuits with n <= 12 pack 2^(12-n)
 * samples into one shared-memory tile; larger ones run window passes of
 * cfgs[0].window qubits (0 = 12) with a per-sample chain of bounded
 * device-side waits (HVP_ETIMEOUT if one expires). With HVP_AUTOTUNE in
 * cfgs[0].flags and a circuit above 12 qubits, the window width is chosen
 * among 12, 11 and 10 by timing the batch at set-up. hvp_plan_info:
 * info[1] = work items, info[2] = window qubits, info[6] = persistent CTAs,
 * info[7] = circuits. */
int hvp_init_batch(hvp_ctx **out, int n_circuits, const hvp_config *cfgs,
                   const double *const *psi_1q, const double *const *ref_data);

/* Test of the batch kernel's bounded device-side waits (no counterpart in the
 * paper). dep_bias = 1 makes every per-sample chain wait ask for one more
 * finished phase than can finish, so the first wait gives up after
 * spin_limit sleeps of 200 ns, every later wait gives up at once, and the
 * next call returns HVP_ETIMEOUT; the context stays usable. dep_bias = 0 with
 * spin_limit = 20000000 restores the normal waits. Applies to the next calls
 * (captured graphs are rebuilt). HVP_EINVAL if ctx is not a batch context,
 * dep_bias is not 0 or 1 or spin_limit < 1. */
int hvp_batch_wait_test(hvp_ctx *ctx, int dep_bias, long long spin_limit);

/* Test of the bounded waits of the forward-cache schedule (no counterpart in
 * the paper). The cached backward kernel waits on an mbarrier for each bulk
 * copy of cached forward states; extra_bytes = 16 makes every such barrier
 * expect 16 bytes more than its copy delivers, so no wait can complete: each
 * gives up after spin_limit polls (0 = the default of 2^23, about two
 * seconds), the kernel stops without writing results, and the next
 * hvp_loss_grad / hvp_hvp call returns HVP_ETIMEOUT; the context stays
 * usable. extra_bytes = 0 with spin_limit = 0 restores normal operation.
 * Applies to the next calls (captured graphs are rebuilt). HVP_EINVAL if the
 * context does not run the forward cache (hvp_plan_info info[3] != 0) or an
 * argument is out of range.
 * On a context with HVP_TENSOR the same call tests the bounded waits of the
 * tensor-core passes: extra_bytes = 16 makes the barrier on which each tile
 * waits for its MMAs expect one arrival more than the MMAs' commit delivers,
 * and limits those waits to spin_limit polls (at least 1); every wait then
 * gives up, the pass commits its MMAs in flight to a separate barrier, waits
 * for them (bounded), frees its tensor memory and stops, and the next call
 * returns HVP_ETIMEOUT. extra_bytes = 0 restores normal operation. */
int hvp_cache_wait_test(hvp_ctx *ctx, int extra_bytes, long long spin_limit);

/* Loss and gradient (Alg. 1 without tangents, Alg. 2 first two steps).
 *   G    : host, K*32 doubles.
 *   loss : host, 1 double (may be NULL).
 *   grad : host, K*32 doubles (may be NULL); Euclidean, or Riemannian with
 *          HVP_RIEMANNIAN.
 * Blocks until the results are on the host. */
int hvp_loss_grad(hvp_ctx *ctx, const double *G, double *loss, double *grad);

/* Loss, gradient and HVP along V in one forward/backward sweep pair
 * (Alg. 1 and Alg. 2; Eq. dfis, dbis, overlap-hvp, hvp-costHS).
 *   G, V : host, K*32 doubles each.
 *   loss, grad, hvp : host outputs (each may be NULL); grad and hvp are
 *          Euclidean, or Riemannian with HVP_RIEMANNIAN.
 * Blocks until the results are on the host. */
int hvp_hvp(hvp_ctx *ctx, const double *G, const double *V, double *loss,
            double *grad, double *hvp);

/* HVPs along n_dir directions at the same gates (Sec. 4: the truncated-CG
 * inner loop and the dense Hessian of App. G evaluate many HVPs at one G).
 * With HVP_MULTI_DIR and the forward cache, directions go through the sweep
 * in pairs: the states psi, the co-states phi and the environments E are
 * computed once per pair and only the tangent states and DE sums per
 * direction (Eq. dfis, Eq. dbis, Eq. Dpsi); an odd last direction, and every
 * direction of other contexts, take one sweep each.
 *   G    : host, K*32 doubles; V : host, n_dir*K*32 doubles (direction d at
 *          offset d*K*32);
 *   loss, grad : host (may be NULL), as for hvp_hvp;
 *   hvp  : host, n_dir*K*32 doubles (may be NULL), Euclidean or Riemannian.
 * Blocks until the results are on the host. */
int hvp_hvp_multi(hvp_ctx *ctx, const double *G, int n_dir, const double *V,
                  double *loss, double *grad, double *hvp);

/* The same on device pointers, stream-ordered on the context's stream. */
int hvp_hvp_multi_dev(hvp_ctx *ctx, const double *G_dev, int n_dir,
                      const double *V_dev, double *loss_dev, double *grad_dev,
                      double *hvp_dev);

/* Stream-ordered variants on device memory (for framework integration):
 * inputs and outputs are device pointers of the same sizes as above; V_dev
 * may be NULL (loss and gradient only); any output may be NULL. Work is
 * enqueued on the context's stream and the call returns without waiting. */
int hvp_hvp_dev(hvp_ctx *ctx, const double *G_dev, const double *V_dev,
                double *loss_dev, double *grad_dev, double *hvp_dev);

/* Results of the last completed call, copied to host memory (synchronises
 * the context's stream):
 *   HVP_OUT_T, HVP_OUT_OMEGA : N_s complex (2*N_s doubles), the overlaps
 *        T_s = phi_s^dagger G psi_s and Omega_s = D T_s[V] (Eq. Omega);
 *   HVP_OUT_GRAD_E, HVP_OUT_HVP_E : Euclidean forms, K*32 doubles;
 *   HVP_OUT_GRAD_R, HVP_OUT_HVP_R : Riemannian forms, K*32 doubles;
 *   HVP_OUT_LOSS : 1 double;
 *   HVP_OUT_ENV : per-sample environments dT_s/dG_k and D(dT_s/dG_k)[V],
 *        N_s*K*32 complex (N_s*K*64 doubles; the 16 entries of E then the
 *        16 of DE per gate); HVP_EINVAL with HVP_TENSOR, whose block
 *        environments are summed over samples. */
#define HVP_OUT_T 1
#define HVP_OUT_OMEGA 2
#define HVP_OUT_GRAD_E 3
#define HVP_OUT_HVP_E 4
#define HVP_OUT_GRAD_R 5
#define HVP_OUT_HVP_R 6
#define HVP_OUT_LOSS 7
#define HVP_OUT_ENV 8
int hvp_get(hvp_ctx *ctx, int what, double *out);

/* Description of the execution plan of a context (host memory):
 *   info[0] = K, info[1] = number of window passes P, info[2] = window
 *   (local qubits per tile), info[3] = checkpoint stride (0: the forward
 *   states before every gate are cached), info[4] = kernel
 *   launches of the last hvp call, info[5] = device memory held by the
 *   context in MiB, info[6] = tiles per CTA, info[7] = CTAs per sample,
 *   info[8] = threads per CTA, info[9] = arithmetic variant.
 * With HVP_TENSOR: info[1] = number of fused blocks, info[2] = 5 (block
 * qubits), info[3] = 0, info[6] = 0, info[7] = CTAs of the backward block
 * passes, info[8] = 256, info[9] = 0 (the tensor-core arithmetic: exact-
 * integer bf16 slice products and TF32 environment products; the window-
 * pass variants are 1 to 3). */
int hvp_plan_info(const hvp_ctx *ctx, long long info[10]);

/* Fused-block plan of the HVP_TENSOR schedule without a context or GPU (for
 * tests and tools): block_of_gate[K] receives the block of each gate and
 * block_qubit[j] the first of block j's five qubits (arrays of K entries,
 * either may be NULL); returns the number of blocks, or HVP_EINVAL for
 * n < 5. */
int hvp_plan_blocks(int n, int n_layers, int *block_of_gate, int *block_qubit);

/* Window-pass plan of a brickwall without a context or GPU (for tests and
 * tools): fills pass_of_gate[K] with the pass index of each gate and returns
 * the number of passes P, or a negative code. window = local qubits per tile
 * (n <= window gives a single pass), low_bits = address bits every tile keeps
 * contiguous. */
int hvp_plan_brickwall(int n, int n_layers, int window, int low_bits, int *pass_of_gate);

/* Runs one evaluation (V_dev NULL: loss and gradient only) launching its
 * kernels one by one with a CUDA event after each launch on the context's
 * stream, and reports per launch: ms[i] the event-to-event device time,
 * kind[i] (HVP_K_* below), flops[i] the algorithmic floating-point
 * operations of that launch (8 per complex multiply-add; per amplitude and
 * gate 12 complex multiply-adds forward and 36 backward with tangents, 4 and
 * 12 without) and bytes[i] its algorithmic HBM bytes (every state element the
 * launch needs read once and every result written once). Arrays hold
 * max_launches entries (host memory).
 * Returns the number of launches (> max_launches: arrays truncated) or a
 * negative code. Synchronises the stream. */
#define HVP_K_PREP 0
#define HVP_K_PASS_FWD 1
#define HVP_K_PASS_TURN 2
#define HVP_K_PASS_BWD 3
#define HVP_K_GATE_INIT 4
#define HVP_K_GATE_FWD 5
#define HVP_K_GATE_PHI 6
#define HVP_K_GATE_BWD 7
#define HVP_K_POST 8
#define HVP_K_BLOCK_FWD 9   /* one fused block applied forward (HVP_TENSOR)   */
#define HVP_K_BLOCK_BWD 10  /* one fused block backward with its environment  */
int hvp_profile(hvp_ctx *ctx, const double *G_dev, const double *V_dev, int max_launches,
                float *ms, int *kind, double *flops, double *bytes);

/* Loss, gradient and HVP without any device allocation, for callers that
 * cannot call cudaMalloc: code running inside a framework that owns the whole
 * device pool through its own allocator, or a host process under a strict
 * device-memory budget. The paper has no counterpart; it is an engineering
 * entry point.
 *
 * The work space is one static device array of HVP_NOALLOC_SCRATCH_BYTES that
 * every GPU which loads this library holds until the process exits. The
 * caller passes all inputs and outputs as device pointers:
 *   psi_1q_dev : N_s*n*4 doubles (as for hvp_init), phi_dev : the reference
 *   states phi_s = U_ref psi_s, N_s * 2^n * 2 doubles in the standard layout;
 *   G_dev, V_dev : K*32 doubles (V_dev NULL: loss and gradient only);
 *   loss_dev (1 double), grad_dev, hvp_dev (K*32 doubles): Euclidean forms;
 *   stream : cudaStream_t (NULL = legacy default stream).
 * Limits: 2 <= n <= 12 (one 2^n tile per sample), K <= 64 gates, and a work
 * space of 2^n*N_s*8 + K*N_s*1024 + K*1680 + N_s*(16n + 32) bytes plus at
 * most 8 kB of tables and alignment, which must fit in
 * HVP_NOALLOC_SCRATCH_BYTES (16 MiB; e.g. n = 12, L = 8, N_s = 128 fits);
 * larger problems return HVP_EINVAL with a message in hvp_last_error(NULL).
 * HVP_ENONFINITE reports a singular or non-finite gate.
 * The call is synchronous: it copies its small tables from host memory into
 * the array, enqueues its kernels on `stream`, reads back a status word and
 * waits for the stream before it returns.
 * The first call on a device also looks up the array's device address.
 * Every call reuses the same array, so
 * calls that overlap on the GPU (other threads, other streams) race; serialise
 * them. */
#define HVP_NOALLOC_SCRATCH_BYTES (16u << 20)
int hvp_hvp_noalloc(int n, int n_layers, int n_samples, const double *psi_1q_dev,
                    const double *phi_dev, const double *G_dev, const double *V_dev,
                    double *loss_dev, double *grad_dev, double *hvp_dev, void *stream);

/* Releases the context and all its device memory; NULL is ignored. */
void hvp_free(hvp_ctx *ctx);

/* Message of the last failed call on ctx, or with ctx == NULL the last
 * failure of hvp_init on the calling thread. Never NULL. */
const char *hvp_last_error(const hvp_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* HVP_H */
