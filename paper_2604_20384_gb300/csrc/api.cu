// C ABI of libhvp: contexts, device memory, the launch schedule of one
// loss/gradient/HVP evaluation and its capture into CUDA graphs.
//
// Schedule of one evaluation on the window-pass path (P passes, Alg. 1):
//   prep (G^-1, G^dag, V^dag in FP64, FP32 copies)
//   forward passes 0 .. P-2, each storing its output states as a checkpoint
//   turnaround pass P-1: forward through its gates, then backward through
//       them with co-states (phi_s, 0)
//   backward passes P-2 .. 0, each reloading the forward checkpoint at its end
//   FP64 post-processing (reduction, T_s, Omega_s, loss, grad, HVP, App. F)
// With a checkpoint stride c > 1 only every c-th boundary is kept and the
// others are recomputed segment by segment before the backward passes need
// them.
//
// Forward-cache schedule (the default when it fits in device memory; Alg. 1
// keeps the forward states of every gate): forward passes 0 .. P-1 also write
// the states before each of their gates into the cache, then backward passes
// P-1 .. 0 read them back (bulk copies into shared memory) instead of
// recomputing them with G^-1 inside each pass. The forward states of the pass
// boundaries are then only needed by the next forward pass (one buffer,
// updated in place).
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/hvp.h"
#include "internal.h"
#include "nvtx.h"

using namespace hvp;

namespace {

thread_local std::string g_init_error;

std::string fmt(const char* f, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, f);
    vsnprintf(buf, sizeof buf, f, ap);
    va_end(ap);
    return buf;
}

}  // namespace

namespace hvp {
// Message returned by hvp_last_error(NULL) on the calling thread.
void set_thread_error(const char* msg) { g_init_error = msg; }
}  // namespace hvp

struct hvp_ctx {
    hvp_config cfg{};
    int K = 0;
    bool dbl = false, unfused = false;
    Plan plan;
    int w = 0, threads = 256, variant = 1, tiles_per_cta = 1, cx_count = 1, stride = 1, P = 0, max_gates = 0;
    int n_slots = 0, s0_last = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<void*> allocs;
    DevPass* d_pass = nullptr;
    DevGate* d_gates = nullptr;
    double2* d_G = nullptr;
    double2* d_V = nullptr;
    void* d_mats = nullptr;
    void* d_psi1q = nullptr;
    void* d_phi = nullptr;
    std::vector<void*> ckpt;   // boundary j -> stored buffer or nullptr
    std::vector<void*> slots;  // recomputed boundaries of one segment
    void* d_scratch = nullptr; // non-stored boundaries of the first forward sweep
    void* d_co = nullptr;      // co-states (a, b)
    bool cache = false;        // forward-cache schedule
    void* d_cache = nullptr;   // K slots of forward states (states before each gate)
    size_t cache_slot = 0;     // bytes of one slot (tangent elements)
    void* d_chain = nullptr;   // forward states between passes (cache schedule)
    unsigned copy_wait_limit = 0, copy_extra_bytes = 0;   // hvp_cache_wait_test
    // two tangent directions per sweep (HVP_MULTI_DIR with the forward cache)
    bool pair = false;
    double2* d_V2 = nullptr;
    void* d_mats2 = nullptr;
    double* d_partial2 = nullptr;
    double* d_env2 = nullptr;
    double* d_res2 = nullptr;
    double* h_res2 = nullptr;
    cudaGraphExec_t gexec_pair = nullptr;
    void* d_x = nullptr;       // unfused forward states
    double* d_partial = nullptr;
    double* d_env = nullptr;
    double* d_res = nullptr;
    int* d_status = nullptr;
    double* h_in = nullptr;
    double* h_res = nullptr;
    int* h_status = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    size_t bytes = 0;
    size_t res_len = 0;
    int launches_per_call[2] = {0, 0};
    std::string err;
    // per-launch profiling (hvp_profile)
    bool prof = false;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_kind;
    std::vector<double> prof_flops, prof_bytes;
    // batched contexts (hvp_init_batch)
    BatchImpl* batch = nullptr;
    int n_circuits = 0;
    // fused-block schedule on the tensor cores (HVP_TENSOR)
    bool tensor = false;
    std::vector<BlockPlan> blocks;
    int nb = 0, tc_ctas_fwd = 1, tc_ctas_bwd = 1, ovl_chunks = 1;
    DevBlock* d_blocks = nullptr;
    DevBlockGate* d_bgates = nullptr;
    Mats64* d_mats64 = nullptr;     // FP64 G, G^-1, V, Y per gate (block post-processing)
    uint32_t* d_ops = nullptr;      // per block: the operator record (integer slices and row scales)
    std::vector<void*> tstate;      // forward states at the output of block j (float4 per amplitude)
    void* d_psi0 = nullptr;         // the product input states (psi, 0), float4 per amplitude
    double* d_rec = nullptr;        // per block and CTA: FP64 environment records (128 x 128)
    double* d_psum = nullptr;       // per block: records summed over CTAs
    double2* d_Ew = nullptr;        // per gate: sum_s conj(T_s) E_s
    double2* d_DEw = nullptr;       // per gate: sum_s conj(Omega_s) E_s + conj(T_s) DE_s
    double* d_ovl = nullptr;        // overlap partial sums
    unsigned tc_wait_limit = 0, tc_barrier_extra = 0;   // hvp_cache_wait_test on a tensor context
    // translation-invariant layers (HVP_TRANSLATION, App. E): the caller's gates
    // and directions are per layer, expanded to every gate on the device, and the
    // per-gate derivative blocks are summed per layer on the device
    bool ti = false;
    double2* d_GL = nullptr;
    double2* d_VL = nullptr;
    int* d_layer_first = nullptr;   // first gate of each layer, n_layers + 1 entries

    size_t off_T() const { return 2; }
    size_t off_Om() const { return 2 + 2 * (size_t)cfg.n_samples; }
    size_t off_ge() const { return 2 + 4 * (size_t)cfg.n_samples; }
    size_t off_he() const { return off_ge() + 32 * (size_t)K; }
    size_t off_gr() const { return off_he() + 32 * (size_t)K; }
    size_t off_hr() const { return off_gr() + 32 * (size_t)K; }
    size_t off_layer() const { return off_hr() + 32 * (size_t)K; }   // [ge, he, gr, hr][n_layers][16] complex
    // the caller's view: 4x4 blocks per call (layers with HVP_TRANSLATION, else gates)
    size_t n_user() const { return ti ? (size_t)cfg.n_layers : (size_t)K; }
    // offsets of the caller's outputs: 0 Euclidean gradient, 1 Euclidean HVP, 2 and 3 Riemannian
    size_t uoff(int i) const {
        if (ti) return off_layer() + (size_t)i * 32 * cfg.n_layers;
        return off_ge() + (size_t)i * 32 * K;
    }
    double2* in_G() const { return ti ? d_GL : d_G; }
    double2* in_V() const { return ti ? d_VL : d_V; }
};

namespace {

int fail(hvp_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    else g_init_error = msg;
    return code;
}

#define CUDA_TRY(ctx, call)                                                                           \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? HVP_ENOMEM : HVP_ECUDA,               \
                        fmt("%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__));   \
    } while (0)

// Records an event after a launch when profiling.
int prof_mark(hvp_ctx* c, int kind, double flops, double bytes) {
    if (!c->prof) return HVP_OK;
    cudaEvent_t e;
    CUDA_TRY(c, cudaEventCreate(&e));
    c->prof_ev.push_back(e);
    CUDA_TRY(c, cudaEventRecord(e, c->stream));
    c->prof_kind.push_back(kind);
    c->prof_flops.push_back(flops);
    c->prof_bytes.push_back(bytes);
    return HVP_OK;
}

int dalloc(hvp_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return HVP_OK;
    if (c->bytes + bytes > device_alloc_cap())
        return fail(c, HVP_ENOMEM, fmt("device allocation of %zu bytes exceeds the cap HVP_DEVICE_ALLOC_CAP_MB "
                                       "(%zu bytes held)", bytes, c->bytes));
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(c, HVP_ENOMEM, fmt("cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e)));
    }
    c->allocs.push_back(*p);
    c->bytes += bytes;
    return HVP_OK;
}

bool all_finite(const double* a, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

size_t state_elt(const hvp_ctx* c) { return c->dbl ? 32 : 16; }   // (psi, dpsi) per amplitude

// ------------------------------------------------------------ tiled schedule

const void* boundary_in(hvp_ctx* c, int j) {   // forward states after pass j-1
    if (j == 0) return nullptr;                // generated in-kernel
    if (c->ckpt[j]) return c->ckpt[j];
    if (j > c->s0_last) return c->slots[j - c->s0_last - 1];
    return c->d_scratch;
}

// cached: a pass of the forward-cache schedule (forward passes write the
// cache, backward passes read it).
int tiled_pass(hvp_ctx* c, int p, int mode, const void* xin, void* xout, bool tan, int ld_out, int st_out,
               const void* mats, const void* phi, bool cached = false) {
    NvtxRange range((mode & M_BWD) ? ((mode & M_FWD) ? "turnaround pass" : "backward pass") : "forward pass", p);
    TiledArgs a{};
    a.pass = c->d_pass + p;
    a.gates = c->d_gates;
    a.mats = reinterpret_cast<const Mats32*>(mats);
    a.psi1q = reinterpret_cast<const float2*>(c->d_psi1q);
    a.xin = xin;
    a.xout = xout;
    a.phi = reinterpret_cast<const float2*>(phi);
    a.cin = c->d_co;
    a.cout = c->d_co;
    a.partial = c->d_partial;
    a.cache = c->d_cache;
    a.cache_slot_bytes = ((size_t)1 << c->cfg.n) * c->cfg.n_samples * (tan ? 16 : 8);
    a.status = c->d_status;
    a.copy_wait_limit = c->copy_wait_limit;
    a.copy_extra_bytes = c->copy_extra_bytes;
    a.n = c->cfg.n;
    a.n_samples = c->cfg.n_samples;
    a.mode = mode;
    a.tiles_per_cta = c->tiles_per_cta;
    a.cx_count = c->cx_count;
    a.ld_out_tab = ld_out;
    a.st_out_tab = st_out;
    const int ng = (int)c->plan.passes[p].gates.size();
    if (cached) CUDA_TRY(c, launch_tiled_cached(a, tan, c->w, c->threads, std::max(ng, 1), c->stream));
    else CUDA_TRY(c, launch_tiled(a, tan, c->w, c->threads, std::max(ng, 1), c->stream, c->variant));
    if (c->prof) {
        // Algorithmic work: 12 (36) complex MACs per amplitude per gate forward
        // (backward) with tangents, 4 (12) without; 8 flops per complex MAC.
        // From the forward cache the backward gate needs 24 (8): the forward
        // states are read, not recomputed, and cost 16 (8) bytes per
        // amplitude per gate, written by the forward pass and read back.
        const double amps = (double)((size_t)1 << c->cfg.n) * c->cfg.n_samples;
        const double elt = tan ? 16.0 : 8.0;
        double fl = 0, by = 0;
        if (mode & M_FWD) fl += amps * ng * (tan ? 96.0 : 32.0);
        if (mode & M_BWD) fl += amps * ng * (cached ? (tan ? 192.0 : 64.0) : (tan ? 288.0 : 96.0));
        if (cached) by += amps * ng * elt;
        if (!(mode & M_GEN) && !(cached && (mode & M_BWD))) by += amps * elt;
        if (mode & M_STORE_F) by += amps * elt;
        if (mode & M_BWD) by += amps * ((mode & M_LOAD_PHI) ? 8.0 : elt);
        if (mode & M_STORE_B) by += amps * elt;
        const int kind = (mode & M_BWD) ? ((mode & M_FWD) ? HVP_K_PASS_TURN : HVP_K_PASS_BWD) : HVP_K_PASS_FWD;
        return prof_mark(c, kind, fl, by);
    }
    return HVP_OK;
}

// Forward-cache schedule: P forward passes filling the cache (the boundary
// states chained in place through d_chain), then P cached backward passes.
int enqueue_cached(hvp_ctx* c, bool tan, int* launches) {
    const int P = c->P;
    int rc, L = 0;
    for (int p = 0; p < P; ++p) {
        const int mode = (p == 0 ? M_GEN : 0) | M_FWD | (p + 1 < P ? M_STORE_F : 0);
        if ((rc = tiled_pass(c, p, mode, p ? c->d_chain : nullptr, c->d_chain, tan, 0, 1, c->d_mats, c->d_phi,
                             true)))
            return rc;
        ++L;
    }
    for (int p = P - 1; p >= 0; --p) {
        const int mode = M_BWD | (p == P - 1 ? M_LOAD_PHI : 0) | (p > 0 ? M_STORE_B : 0);
        if ((rc = tiled_pass(c, p, mode, nullptr, nullptr, tan, 1, 0, c->d_mats, c->d_phi, true))) return rc;
        ++L;
    }
    *launches = L;
    return HVP_OK;
}

int enqueue_tiled(hvp_ctx* c, bool tan, int* launches) {
    if (c->cache) return enqueue_cached(c, tan, launches);
    const int P = c->P, cs = c->stride;
    int rc, L = 0;
    // First forward sweep.
    for (int p = 0; p + 1 < P; ++p) {
        const int j = p + 1;
        void* out = c->ckpt[j] ? c->ckpt[j] : (j > c->s0_last ? c->slots[j - c->s0_last - 1] : c->d_scratch);
        const int mode = (p == 0 ? M_GEN : 0) | M_FWD | M_STORE_F;
        if ((rc = tiled_pass(c, p, mode, boundary_in(c, p), out, tan, 0, 1, c->d_mats, c->d_phi))) return rc;
        ++L;
    }
    // Backward, segment by segment from the end.
    const int nseg = (P - 1) / cs + 1;
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int s0 = sg * cs, s1 = std::min(s0 + cs, P);
        if (s0 != c->s0_last) {   // recompute boundaries s0+1 .. s1-1 into the slots
            for (int p = s0; p + 1 < s1; ++p) {
                const void* in = p == s0 ? boundary_in(c, s0) : c->slots[p - s0 - 1];
                const int mode = (p == 0 ? M_GEN : 0) | M_FWD | M_STORE_F;
                if ((rc = tiled_pass(c, p, mode, in, c->slots[p - s0], tan, 0, 1, c->d_mats, c->d_phi))) return rc;
                ++L;
            }
        }
        for (int p = s1 - 1; p >= s0; --p) {
            if (p == P - 1) {
                const int mode = (P == 1 ? M_GEN : 0) | M_FWD | M_BWD | M_LOAD_PHI | (P > 1 ? M_STORE_B : 0);
                const void* in = boundary_in(c, P - 1);
                if ((rc = tiled_pass(c, p, mode, in, nullptr, tan, 0, 0, c->d_mats, c->d_phi))) return rc;
            } else {
                const void* in = (p + 1 == s1) ? c->ckpt[s1] : c->slots[p - s0];
                const int mode = M_BWD | (p > 0 ? M_STORE_B : 0);
                if ((rc = tiled_pass(c, p, mode, in, nullptr, tan, 1, 0, c->d_mats, c->d_phi))) return rc;
            }
            ++L;
        }
    }
    *launches = L;
    return HVP_OK;
}

int enqueue_unfused(hvp_ctx* c, bool tan, int* launches) {
    const int n = c->cfg.n, ns = c->cfg.n_samples, K = c->K;
    int L = 0;
    const double amps = (double)((size_t)1 << n) * ns;
    const double cb = c->dbl ? 16.0 : 8.0, elt = (tan ? 2.0 : 1.0) * cb;
    int rc;
    CUDA_TRY(c, unfused_init(c->dbl, c->d_psi1q, c->d_x, n, ns, tan, c->stream));
    if ((rc = prof_mark(c, HVP_K_GATE_INIT, 0.0, amps * elt))) return rc;
    ++L;
    for (int k = 0; k < K; ++k) {
        NvtxRange range("forward gate", k);
        CUDA_TRY(c, unfused_fwd_gate(c->dbl, c->d_mats, k, c->plan.first_qubit[k], c->d_x, n, ns, tan, c->stream));
        if ((rc = prof_mark(c, HVP_K_GATE_FWD, amps * (tan ? 96.0 : 32.0), 2 * amps * elt))) return rc;
        ++L;
    }
    CUDA_TRY(c, unfused_load_phi(c->dbl, c->d_phi, c->d_co, n, ns, tan, c->stream));
    if ((rc = prof_mark(c, HVP_K_GATE_PHI, 0.0, amps * (cb + elt)))) return rc;
    ++L;
    for (int k = K - 1; k >= 0; --k) {
        NvtxRange range("backward gate", k);
        CUDA_TRY(c, unfused_bwd_gate(c->dbl, c->d_mats, k, c->plan.first_qubit[k], c->d_x, c->d_co, c->d_partial, n,
                                     ns, c->cx_count, tan, c->stream));
        if ((rc = prof_mark(c, HVP_K_GATE_BWD, amps * (tan ? 288.0 : 96.0), 4 * amps * elt))) return rc;
        ++L;
    }
    *launches = L;
    return HVP_OK;
}

// One pass of the two-direction schedule (both directions' tangents in one
// sweep, forward cache of 24 bytes per amplitude per gate).
int pair_pass(hvp_ctx* c, int p, int mode) {
    NvtxRange range((mode & M_BWD) ? ((mode & M_FWD) ? "turnaround pass" : "backward pass") : "forward pass", p);
    TiledArgs a{};
    a.pass = c->d_pass + p;
    a.gates = c->d_gates;
    a.mats = reinterpret_cast<const Mats32*>(c->d_mats);
    a.mats2 = reinterpret_cast<const Mats32*>(c->d_mats2);
    a.psi1q = reinterpret_cast<const float2*>(c->d_psi1q);
    a.xin = c->d_chain;
    a.xout = c->d_chain;
    a.phi = reinterpret_cast<const float2*>(c->d_phi);
    a.cin = c->d_co;
    a.cout = c->d_co;
    a.partial = c->d_partial;
    a.partial2 = c->d_partial2;
    a.cache = c->d_cache;
    a.cache_slot_bytes = ((size_t)1 << c->cfg.n) * c->cfg.n_samples * 24;
    a.status = c->d_status;
    a.copy_wait_limit = c->copy_wait_limit;
    a.copy_extra_bytes = c->copy_extra_bytes;
    a.n = c->cfg.n;
    a.n_samples = c->cfg.n_samples;
    a.mode = mode;
    a.tiles_per_cta = c->tiles_per_cta;
    a.cx_count = c->cx_count;
    const int ng = (int)c->plan.passes[p].gates.size();
    CUDA_TRY(c, launch_pair(a, c->w, std::max(ng, 1), c->stream));
    return HVP_OK;
}

PostArgs post_args(hvp_ctx* c, double* partial, double* env, const double2* V, double* res) {
    PostArgs p{};
    p.partial = partial;
    p.env = env;
    p.G = c->d_G;
    p.V = V;
    p.T = reinterpret_cast<double2*>(res + c->off_T());
    p.Omega = reinterpret_cast<double2*>(res + c->off_Om());
    p.loss = res;
    p.grad_e = reinterpret_cast<double2*>(res + c->off_ge());
    p.hvp_e = reinterpret_cast<double2*>(res + c->off_he());
    p.grad_r = reinterpret_cast<double2*>(res + c->off_gr());
    p.hvp_r = reinterpret_cast<double2*>(res + c->off_hr());
    p.K = c->K;
    p.n_samples = c->cfg.n_samples;
    p.cx_count = c->cx_count;
    p.tangent = 1;
    p.frobenius = (c->cfg.flags & HVP_FROBENIUS) ? 1 : 0;
    return p;
}

// Loss, gradient and the HVPs along d_V and d_V2 in one sweep pair: results
// of direction 1 in d_res, of direction 2 in d_res2.
int enqueue_pair(hvp_ctx* c) {
    int rc;
    const int P = c->P;
    CUDA_TRY(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    CUDA_TRY(c, launch_prep(c->d_G, c->d_V, c->d_mats, false, c->K, c->d_status, c->stream));
    CUDA_TRY(c, launch_prep(c->d_G, c->d_V2, c->d_mats2, false, c->K, c->d_status, c->stream));
    for (int p = 0; p < P; ++p)
        if ((rc = pair_pass(c, p, (p == 0 ? M_GEN : 0) | M_FWD | (p + 1 < P ? M_STORE_F : 0)))) return rc;
    for (int p = P - 1; p >= 0; --p)
        if ((rc = pair_pass(c, p, M_BWD | (p == P - 1 ? M_LOAD_PHI : 0) | (p > 0 ? M_STORE_B : 0)))) return rc;
    CUDA_TRY(c, launch_post(post_args(c, c->d_partial, c->d_env, c->d_V, c->d_res), c->stream));
    CUDA_TRY(c, launch_post(post_args(c, c->d_partial2, c->d_env2, c->d_V2, c->d_res2), c->stream));
    return HVP_OK;
}

int run_pair(hvp_ctx* c) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CUDA_TRY(c, cudaStreamIsCapturing(c->stream, &cap));
    if ((c->cfg.flags & HVP_NO_GRAPH) || cap != cudaStreamCaptureStatusNone) return enqueue_pair(c);
    if (!c->gexec_pair) {
        cudaGraph_t g = nullptr;
        CUDA_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_pair(c);
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return fail(c, HVP_ECUDA, fmt("graph capture failed: %s", cudaGetErrorString(e)));
        e = cudaGraphInstantiate(&c->gexec_pair, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->gexec_pair = nullptr;
            return fail(c, HVP_ECUDA, fmt("graph instantiation failed: %s", cudaGetErrorString(e)));
        }
    }
    CUDA_TRY(c, cudaGraphLaunch(c->gexec_pair, c->stream));
    return HVP_OK;
}

// Fused-block schedule (HVP_TENSOR): FP64 gate and block preparation, the
// forward block passes keeping the states at every block boundary, the
// overlaps T_s, Omega_s, the backward block passes from the weighted
// co-states (T_s phi_s, Omega_s phi_s) accumulating the block environments,
// and the FP64 reduction to per-gate gradient and HVP blocks.
int enqueue_tensor(hvp_ctx* c, bool tan) {
    const int n = c->cfg.n, ns = c->cfg.n_samples, nb = c->nb;
    const bool frob = (c->cfg.flags & HVP_FROBENIUS) != 0;
    const double amps = (double)((size_t)1 << n) * ns;
    const long long ncols = (long long)ns << (n - 5);
    double2* T = reinterpret_cast<double2*>(c->d_res + c->off_T());
    double2* Om = reinterpret_cast<double2*>(c->d_res + c->off_Om());
    int rc, L = 0;
    CUDA_TRY(c, launch_prep(c->d_G, tan ? c->d_V : nullptr, c->d_mats64, true, c->K, c->d_status, c->stream));
    CUDA_TRY(c, launch_block_prep(c->d_blocks, c->d_bgates, nb, c->d_G, tan ? c->d_V : nullptr, c->d_ops,
                                  c->d_status, c->stream));
    if ((rc = prof_mark(c, HVP_K_PREP, 0.0, 0.0))) return rc;
    L += 2;
    // Tensor-pipe flops per amplitude and block: forward, two halves of the
    // 128 x 64 operator x 4 components / 32 amplitudes, six bf16 slice
    // products each (6144; half of it without tangents); backward, plus the
    // environment GEMM, 128 x 128 x 4 / 32 with three TF32 products (3072).
    const double fl_fwd = tan ? 6144.0 : 3072.0, fl_bwd = fl_fwd + 3072.0;
    for (int j = 0; j < nb; ++j) {
        TcbArgs a{};
        a.ops = c->d_ops + (size_t)j * kOpWords;
        a.xin = reinterpret_cast<const float4*>(j ? c->tstate[j - 1] : c->d_psi0);
        a.xout = reinterpret_cast<float4*>(c->tstate[j]);
        a.status = c->d_status;
        a.ncols = ncols;
        a.n = n;
        a.a = c->blocks[j].a;
        a.mode = tan ? 0 : TCB_NO_TANGENT;
        a.wait_limit = c->tc_wait_limit;
        a.barrier_extra = c->tc_barrier_extra;
        NvtxRange range("forward block", j);
        CUDA_TRY(c, launch_tcb(a, false, c->tc_ctas_fwd, c->stream));
        if ((rc = prof_mark(c, HVP_K_BLOCK_FWD, amps * fl_fwd, amps * 32.0))) return rc;
        ++L;
    }
    CUDA_TRY(c, launch_overlaps(reinterpret_cast<const float4*>(c->tstate[nb - 1]),
                                reinterpret_cast<const float2*>(c->d_phi), c->d_ovl, T, Om, n, ns, c->ovl_chunks,
                                c->stream));
    if ((rc = prof_mark(c, HVP_K_POST, 0.0, amps * 24.0))) return rc;
    L += 2;
    // the co-states entering the backward sweep, weighted by the overlaps
    CUDA_TRY(c, launch_weighted_phi(reinterpret_cast<const float2*>(c->d_phi), frob ? nullptr : T, frob ? nullptr : Om,
                                    reinterpret_cast<float4*>(c->d_co), n, ns, c->stream));
    if ((rc = prof_mark(c, HVP_K_POST, 0.0, amps * 24.0))) return rc;
    ++L;
    for (int j = nb - 1; j >= 0; --j) {
        TcbArgs a{};
        a.ops = c->d_ops + (size_t)j * kOpWords;
        a.xin = reinterpret_cast<const float4*>(c->d_co);
        a.xout = reinterpret_cast<float4*>(c->d_co);
        a.psi = reinterpret_cast<const float4*>(j ? c->tstate[j - 1] : c->d_psi0);
        a.rec = c->d_rec + (size_t)j * c->tc_ctas_bwd * 16384;
        a.status = c->d_status;
        a.ncols = ncols;
        a.n = n;
        a.a = c->blocks[j].a;
        a.mode = (j == 0 ? TCB_NO_STORE : 0) | (tan ? 0 : TCB_NO_TANGENT);
        a.wait_limit = c->tc_wait_limit;
        a.barrier_extra = c->tc_barrier_extra;
        NvtxRange range("backward block", j);
        CUDA_TRY(c, launch_tcb(a, true, c->tc_ctas_bwd, c->stream));
        const double by = 32.0 + (j ? 16.0 : 0.0);
        if ((rc = prof_mark(c, HVP_K_BLOCK_BWD, amps * fl_bwd, amps * by))) return rc;
        ++L;
    }
    CUDA_TRY(c, launch_block_post(c->d_blocks, c->d_bgates, nb, c->d_rec, c->tc_ctas_bwd, c->d_psum, c->d_mats64,
                                  c->d_Ew, c->d_DEw, tan ? 1 : 0, c->stream));
    CUDA_TRY(c, launch_post_weighted(c->d_Ew, c->d_DEw, c->d_G, c->d_V, T,
                                     reinterpret_cast<double2*>(c->d_res + c->off_ge()),
                                     reinterpret_cast<double2*>(c->d_res + c->off_he()),
                                     reinterpret_cast<double2*>(c->d_res + c->off_gr()),
                                     reinterpret_cast<double2*>(c->d_res + c->off_hr()), c->d_res, c->K, ns,
                                     tan ? 1 : 0, frob ? 1 : 0, c->stream));
    if ((rc = prof_mark(c, HVP_K_POST, 0.0, 0.0))) return rc;
    L += 4;
    c->launches_per_call[tan ? 1 : 0] = L;   // kernels (the status reset is a memset)
    return HVP_OK;
}

int enqueue_all(hvp_ctx* c, bool tan) {
    int L = 0, rc;
    CUDA_TRY(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    if (c->ti)
        CUDA_TRY(c, launch_expand_layers(c->d_GL, tan ? c->d_VL : nullptr, c->d_G, c->d_V, c->d_layer_first,
                                         c->cfg.n_layers, c->stream));
    if (c->tensor) {
        if ((rc = enqueue_tensor(c, tan))) return rc;
        if (c->ti) {
            CUDA_TRY(c, launch_contract_layers(reinterpret_cast<const double2*>(c->d_res + c->off_ge()),
                                               reinterpret_cast<double2*>(c->d_res + c->off_layer()),
                                               c->d_layer_first, c->cfg.n_layers, c->K, c->stream));
            c->launches_per_call[tan ? 1 : 0] += 2;   // the layer expansion and contraction
        }
        return HVP_OK;
    }
    CUDA_TRY(c, launch_prep(c->d_G, tan ? c->d_V : nullptr, c->d_mats, c->dbl, c->K, c->d_status, c->stream));
    if ((rc = prof_mark(c, HVP_K_PREP, 0.0, 0.0))) return rc;
    ++L;
    int Ls = 0;
    rc = c->unfused ? enqueue_unfused(c, tan, &Ls) : enqueue_tiled(c, tan, &Ls);
    if (rc) return rc;
    L += Ls;
    PostArgs p{};
    p.partial = c->d_partial;
    p.env = c->d_env;
    p.G = c->d_G;
    p.V = c->d_V;
    p.T = reinterpret_cast<double2*>(c->d_res + c->off_T());
    p.Omega = reinterpret_cast<double2*>(c->d_res + c->off_Om());
    p.loss = c->d_res;
    p.grad_e = reinterpret_cast<double2*>(c->d_res + c->off_ge());
    p.hvp_e = reinterpret_cast<double2*>(c->d_res + c->off_he());
    p.grad_r = reinterpret_cast<double2*>(c->d_res + c->off_gr());
    p.hvp_r = reinterpret_cast<double2*>(c->d_res + c->off_hr());
    p.K = c->K;
    p.n_samples = c->cfg.n_samples;
    p.cx_count = c->cx_count;
    p.tangent = tan ? 1 : 0;
    p.frobenius = (c->cfg.flags & HVP_FROBENIUS) ? 1 : 0;
    CUDA_TRY(c, launch_post(p, c->stream));
    if (c->ti)
        CUDA_TRY(c, launch_contract_layers(reinterpret_cast<const double2*>(c->d_res + c->off_ge()),
                                           reinterpret_cast<double2*>(c->d_res + c->off_layer()),
                                           c->d_layer_first, c->cfg.n_layers, c->K, c->stream));
    if ((rc = prof_mark(c, HVP_K_POST, 0.0, 0.0))) return rc;
    L += 4 + (c->ti ? 2 : 0);
    c->launches_per_call[tan ? 1 : 0] = L;
    return HVP_OK;
}

// Runs one evaluation on the context's stream: replays the captured graph, or
// launches directly when graphs are off or the stream is already capturing.
int run(hvp_ctx* c, bool tan) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CUDA_TRY(c, cudaStreamIsCapturing(c->stream, &cap));
    if ((c->cfg.flags & HVP_NO_GRAPH) || cap != cudaStreamCaptureStatusNone) return enqueue_all(c, tan);
    cudaGraphExec_t& ge = c->gexec[tan ? 1 : 0];
    if (!ge) {
        cudaGraph_t g = nullptr;
        CUDA_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_all(c, tan);
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return fail(c, HVP_ECUDA, fmt("graph capture failed: %s", cudaGetErrorString(e)));
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ge = nullptr;
            return fail(c, HVP_ECUDA, fmt("graph instantiation failed: %s", cudaGetErrorString(e)));
        }
    }
    CUDA_TRY(c, cudaGraphLaunch(ge, c->stream));
    return HVP_OK;
}

int compute_phi_from_uref(hvp_ctx* c, const double* uref) {
    const int n = c->cfg.n, ns = c->cfg.n_samples;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_G, uref, 32 * sizeof(double) * c->K, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    if (c->tensor) {
        // the forward block passes without tangents (the block operators of U_ref
        // with dB = 0), then the states of the last boundary into phi
        CUDA_TRY(c, launch_prep(c->d_G, nullptr, c->d_mats64, true, c->K, c->d_status, c->stream));
        CUDA_TRY(c, launch_block_prep(c->d_blocks, c->d_bgates, c->nb, c->d_G, nullptr, c->d_ops, c->d_status,
                                      c->stream));
        for (int j = 0; j < c->nb; ++j) {
            TcbArgs a{};
            a.ops = c->d_ops + (size_t)j * kOpWords;
            a.xin = reinterpret_cast<const float4*>(j ? c->tstate[j - 1] : c->d_psi0);
            a.xout = reinterpret_cast<float4*>(c->tstate[j]);
            a.status = c->d_status;
            a.ncols = (long long)ns << (n - 5);
            a.n = n;
            a.a = c->blocks[j].a;
            a.mode = TCB_NO_TANGENT;
            CUDA_TRY(c, launch_tcb(a, false, c->tc_ctas_fwd, c->stream));
        }
        CUDA_TRY(c, launch_extract_psi(reinterpret_cast<const float4*>(c->tstate[c->nb - 1]),
                                       reinterpret_cast<float2*>(c->d_phi), ((size_t)1 << n) * ns, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        if (*c->h_status & 2) return fail(c, HVP_ETIMEOUT, "a bounded wait of a tensor-core pass expired");
        if (*c->h_status) return fail(c, HVP_ENONFINITE, "U_ref contains a non-finite or singular gate");
        return HVP_OK;
    }
    CUDA_TRY(c, launch_prep(c->d_G, nullptr, c->d_mats, c->dbl, c->K, c->d_status, c->stream));
    if (c->unfused) {
        CUDA_TRY(c, unfused_init(c->dbl, c->d_psi1q, c->d_phi, n, ns, false, c->stream));
        for (int k = 0; k < c->K; ++k)
            CUDA_TRY(c, unfused_fwd_gate(c->dbl, c->d_mats, k, c->plan.first_qubit[k], c->d_phi, n, ns, false,
                                         c->stream));
    } else {
        // psi-only forward passes, in place on the phi buffer; the result ends in
        // the layout of the last pass, which is where the turnaround pass reads it.
        for (int p = 0; p < c->P; ++p) {
            const int mode = (p == 0 ? M_GEN : 0) | M_FWD | M_STORE_F;
            int rc = tiled_pass(c, p, mode, c->d_phi, c->d_phi, false, 0, 1, c->d_mats, nullptr);
            if (rc) return rc;
        }
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (*c->h_status) return fail(c, HVP_ENONFINITE, "U_ref contains a non-finite or singular gate");
    return HVP_OK;
}

// Tiles per CTA: about eight waves of CTAs over 152 SMs, every CTA on tiles of
// one sample (its environment sums are per sample).
int choose_tiling(hvp_ctx* c) {
    const int ns = c->cfg.n_samples;
    const long long tps = 1ll << (c->cfg.n - c->w);
    // About 16 waves of resident CTAs (one per SM at 256 or 512 threads, two
    // at 128): the last, partly filled wave then costs a few percent of a
    // launch at most (measured on GB300 at n = 20, N_s = 64: 8 waves 97.3 ms,
    // 16 waves 94.6 ms, 32 waves 94.8 ms per evaluation). More CTAs per
    // sample also means more FP64 environment records to reduce.
    const long long per_sm = c->threads <= 128 ? 2 : 1;
    long long cx = 1;
    while (cx < tps && cx * ns < 16 * 152 * per_sm) cx *= 2;
    c->cx_count = (int)cx;
    c->tiles_per_cta = (int)(tps / cx);
    return HVP_OK;
}

int init_impl(hvp_ctx* c, const hvp_config* cfg, const double* psi_1q, const double* ref) {
    if (!cfg || !psi_1q || !ref) return fail(c, HVP_EINVAL, "hvp_init: NULL argument");
    c->cfg = *cfg;
    const int n = cfg->n, L = cfg->n_layers, ns = cfg->n_samples;
    if (n < 2 || n > kMaxN) return fail(c, HVP_EINVAL, fmt("n = %d outside [2, %d]", n, kMaxN));
    if (L < 1) return fail(c, HVP_EINVAL, "n_layers must be >= 1");
    if (ns < 1) return fail(c, HVP_EINVAL, "n_samples must be >= 1");
    if (ns > kMaxSamples)   // one grid row per sample in the window-pass launches
        return fail(c, HVP_EINVAL, fmt("n_samples = %d above %d", ns, kMaxSamples));
    if (cfg->precision != HVP_C64 && cfg->precision != HVP_C128) return fail(c, HVP_EINVAL, "unknown precision");
    if (cfg->flags &
        ~(HVP_RIEMANNIAN | HVP_PHI_GIVEN | HVP_UNFUSED | HVP_NO_GRAPH | HVP_AUTOTUNE | HVP_FROBENIUS | HVP_RECOMPUTE |
          HVP_MULTI_DIR | HVP_TENSOR | HVP_TRANSLATION))
        return fail(c, HVP_EINVAL, "unknown flag bits");
    if ((cfg->flags & HVP_TRANSLATION) && (cfg->flags & HVP_MULTI_DIR))
        return fail(c, HVP_EINVAL, "HVP_TRANSLATION cannot be combined with HVP_MULTI_DIR");
    if ((cfg->flags & HVP_TENSOR) &&
        (cfg->precision != HVP_C64 || (cfg->flags & (HVP_UNFUSED | HVP_MULTI_DIR | HVP_RECOMPUTE)) || n < 5))
        return fail(c, HVP_EINVAL, "HVP_TENSOR needs complex64, n >= 5 and none of HVP_UNFUSED, HVP_MULTI_DIR, "
                                   "HVP_RECOMPUTE");
    if (cfg->checkpoint_stride < 0) return fail(c, HVP_EINVAL, "checkpoint_stride must be >= 0");
    if (cfg->window != 0 && (cfg->window < 6 || cfg->window > 12))
        return fail(c, HVP_EINVAL, "window must be 0 (auto) or in [6, 12]");
    if ((cfg->flags & HVP_MULTI_DIR) && cfg->window > 11)
        return fail(c, HVP_EINVAL, "HVP_MULTI_DIR needs a window of at most 11 qubits (two-direction tiles)");
    if (cfg->threads != 0 && cfg->threads != 128 && cfg->threads != 256 && cfg->threads != 512)
        return fail(c, HVP_EINVAL, "threads must be 0 (auto), 128, 256 or 512");
    if (cfg->variant < 0 || cfg->variant > 3) return fail(c, HVP_EINVAL, "variant must be 0 (auto), 1, 2 or 3");
    if (cfg->threads == 128 && cfg->variant > 1)
        return fail(c, HVP_EINVAL, "128 threads run the scalar arithmetic (variant 0 or 1) only");
    if (((size_t)1 << n) * (size_t)ns > ((size_t)1 << 34))
        return fail(c, HVP_EINVAL, "2^n * n_samples above 2^34 amplitudes");
    if (!all_finite(psi_1q, (size_t)ns * n * 4)) return fail(c, HVP_ENONFINITE, "psi_1q is not finite");
    c->K = num_gates(n, L);
    c->dbl = cfg->precision == HVP_C128;
    c->unfused = c->dbl || (cfg->flags & HVP_UNFUSED);
    const size_t dim = (size_t)1 << n;
    if (cfg->flags & HVP_PHI_GIVEN) {
        if (!all_finite(ref, dim * ns * 2)) return fail(c, HVP_ENONFINITE, "phi is not finite");
    } else if (!all_finite(ref, 32 * (size_t)c->K)) {
        return fail(c, HVP_ENONFINITE, "U_ref is not finite");
    }

    CUDA_TRY(c, cudaSetDevice(cfg->device));
    if (cfg->stream) {
        c->stream = (cudaStream_t)cfg->stream;
    } else {
        CUDA_TRY(c, cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }

    // Autotuning: time each (window, arithmetic) candidate with a temporary
    // context and keep the fastest (identity gates: the cost of a sweep does
    // not depend on the gate values).
    hvp_config tuned = *cfg;
    if ((cfg->flags & HVP_AUTOTUNE) && !c->unfused) {
        std::vector<int> windows;
        for (int wdw : {12, 11, 10})
            if ((wdw <= n || windows.empty()) && !((cfg->flags & HVP_MULTI_DIR) && wdw > 11))
                windows.push_back(std::min(wdw, n));
        std::sort(windows.begin(), windows.end());
        windows.erase(std::unique(windows.begin(), windows.end()), windows.end());
        std::vector<double> eye(32 * (size_t)c->K, 0.0), res_g(32 * (size_t)c->K), res_h(32 * (size_t)c->K);
        for (int k = 0; k < c->K; ++k)
            for (int d = 0; d < 4; ++d) eye[32 * (size_t)k + 2 * (d * 4 + d)] = 1.0;
        double best = 1e300;
        // candidates: (window, threads, arithmetic, recompute); 128-thread
        // CTAs pair up on one SM when the window's tiles leave room in shared
        // memory; recompute = 0 is the forward-cache schedule (scalar
        // arithmetic), which a candidate context takes when the cache fits
        std::vector<std::array<int, 4>> cands;
        const bool may_cache = !(cfg->flags & HVP_RECOMPUTE) && cfg->checkpoint_stride == 0;
        for (int wdw : windows) {
            for (int var : {1, 2, 3}) cands.push_back({wdw, 256, var, 1});
            if (wdw <= 11) cands.push_back({wdw, 128, 1, 1});
            if (may_cache) {
                cands.push_back({wdw, 256, 1, 0});
                if (wdw <= 11) cands.push_back({wdw, 128, 1, 0});
            }
        }
        // the fused-block tensor-core schedule (taken when its states fit)
        const bool may_tensor = !(cfg->flags & (HVP_MULTI_DIR | HVP_RECOMPUTE)) && cfg->checkpoint_stride == 0 && n >= 5;
        if (may_tensor) cands.push_back({0, 256, 0, 2});
        for (const auto& cand : cands) {
            const int wdw = cand[0], var = cand[2];
            hvp_config sc = *cfg;
            sc.flags &= ~(HVP_AUTOTUNE | HVP_TENSOR | HVP_TRANSLATION);
            if (cand[3] == 1) sc.flags |= HVP_RECOMPUTE;
            if (cand[3] == 2) sc.flags |= HVP_TENSOR;
            sc.window = wdw >= n ? 0 : wdw;
            sc.threads = cand[1];
            sc.variant = var;
            hvp_ctx* tmp = nullptr;
            if (hvp_init(&tmp, &sc, psi_1q, ref) != HVP_OK) continue;
            double loss = 0.0;
            int ok = hvp_hvp(tmp, eye.data(), eye.data(), &loss, res_g.data(), res_h.data());
            auto t0 = std::chrono::steady_clock::now();
            for (int r = 0; r < 2 && ok == HVP_OK; ++r)
                ok = hvp_hvp(tmp, eye.data(), eye.data(), &loss, res_g.data(), res_h.data());
            const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            hvp_free(tmp);
            if (ok == HVP_OK && dt < best) {
                best = dt;
                tuned.window = sc.window;
                tuned.threads = sc.threads;
                tuned.variant = var;
                tuned.flags = (cfg->flags & ~(HVP_RECOMPUTE | HVP_TENSOR)) | (sc.flags & (HVP_RECOMPUTE | HVP_TENSOR));
            }
        }
        cudaGetLastError();
        c->cfg.flags = (c->cfg.flags & ~(HVP_RECOMPUTE | HVP_TENSOR)) | (tuned.flags & (HVP_RECOMPUTE | HVP_TENSOR));
    }
    c->tensor = (c->cfg.flags & HVP_TENSOR) != 0;

    // Plan.
    int rc;
    if (c->tensor) {
        CUDA_TRY(c, tcb_set_smem_limits());
        if ((rc = make_block_plan(n, L, c->blocks))) return fail(c, rc, "block planning failed");
        brickwall_layout(n, L, c->plan.first_qubit);
        c->plan.n = n; c->plan.L = L; c->plan.K = c->K;
        c->nb = (int)c->blocks.size();
        c->P = 0;
        int sms = 152;
        CUDA_TRY(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cfg->device));
        const long long ncols = (long long)ns << (n - 5);
        c->tc_ctas_fwd = std::max(1, std::min(sms, tcb_tiles(ncols, false)));
        c->tc_ctas_bwd = std::max(1, std::min(sms, tcb_tiles(ncols, true)));
        c->ovl_chunks = (int)std::max<long long>(1, std::min<long long>(((long long)1 << n) / 4096, (4 * sms + ns - 1) / ns));
    } else if (c->unfused) {
        brickwall_layout(n, L, c->plan.first_qubit);
        c->plan.n = n; c->plan.L = L; c->plan.K = c->K;
        c->cx_count = unfused_cx_count(n, ns);
        c->P = 0;
    } else {
        CUDA_TRY(c, tiled_set_smem_limits());
        c->w = std::min(n, tuned.window ? tuned.window : ((cfg->flags & HVP_MULTI_DIR) ? 11 : 12));
        c->threads = tuned.threads ? tuned.threads : 256;
        c->variant = tuned.variant ? tuned.variant : 1;
        if ((rc = make_plan(n, L, c->w, std::min(kLowBits, c->w - 1), c->plan))) return fail(c, rc, "planning failed");
        c->P = (int)c->plan.passes.size();
        for (auto& pp : c->plan.passes) c->max_gates = std::max(c->max_gates, (int)pp.gates.size());
        choose_tiling(c);
    }

    // Device memory.
    const size_t ctype = c->dbl ? 16 : 8;
    if ((rc = dalloc(c, (void**)&c->d_G, 16 * 16 * (size_t)c->K))) return rc;
    if ((rc = dalloc(c, (void**)&c->d_V, 16 * 16 * (size_t)c->K))) return rc;
    if ((rc = dalloc(c, &c->d_mats, (c->dbl ? sizeof(Mats64) : sizeof(Mats32)) * (size_t)c->K))) return rc;
    if ((rc = dalloc(c, &c->d_psi1q, ctype * 2 * (size_t)n * ns))) return rc;
    if ((rc = dalloc(c, &c->d_phi, ctype * dim * ns))) return rc;
    const bool multi = (cfg->flags & HVP_MULTI_DIR) && !c->unfused;
    // two-direction sweeps keep (phi, dphi_1, dphi_2): 24 bytes per amplitude
    if ((rc = dalloc(c, &c->d_co, (multi ? 24 : state_elt(c)) * dim * ns))) return rc;
    if ((rc = dalloc(c, (void**)&c->d_partial, 64 * sizeof(double) * (size_t)c->K * ns * c->cx_count))) return rc;
    if ((rc = dalloc(c, (void**)&c->d_env, 64 * sizeof(double) * (size_t)c->K * ns))) return rc;
    c->ti = (cfg->flags & HVP_TRANSLATION) != 0;
    c->res_len = c->off_layer() + (c->ti ? 4 * 32 * (size_t)L : 0);
    if (c->ti) {
        std::vector<int> first(L + 1, 0);
        for (int l = 0; l < L; ++l) first[l + 1] = first[l] + (n - l % 2) / 2;
        if ((rc = dalloc(c, (void**)&c->d_GL, 16 * 16 * (size_t)L))) return rc;
        if ((rc = dalloc(c, (void**)&c->d_VL, 16 * 16 * (size_t)L))) return rc;
        if ((rc = dalloc(c, (void**)&c->d_layer_first, sizeof(int) * (L + 1)))) return rc;
        CUDA_TRY(c, cudaMemcpy(c->d_layer_first, first.data(), sizeof(int) * (L + 1), cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemset(c->d_VL, 0, 16 * 16 * (size_t)L));
    }
    if ((rc = dalloc(c, (void**)&c->d_res, sizeof(double) * c->res_len))) return rc;
    if ((rc = dalloc(c, (void**)&c->d_status, sizeof(int)))) return rc;
    CUDA_TRY(c, cudaMemset(c->d_V, 0, 16 * 16 * (size_t)c->K));
    CUDA_TRY(c, cudaMemset(c->d_res, 0, sizeof(double) * c->res_len));
    CUDA_TRY(c, cudaMallocHost((void**)&c->h_in, sizeof(double) * 64 * (size_t)c->K));
    CUDA_TRY(c, cudaMallocHost((void**)&c->h_res, sizeof(double) * c->res_len));
    CUDA_TRY(c, cudaMallocHost((void**)&c->h_status, sizeof(int)));

    if (c->tensor) {
        std::vector<DevBlock> db;
        std::vector<DevBlockGate> dbg;
        for (const BlockPlan& bp : c->blocks) {
            db.push_back(DevBlock{bp.a, (int)bp.gates.size(), (int)dbg.size(), 0});
            for (int k : bp.gates) dbg.push_back(DevBlockGate{k, c->plan.first_qubit[k] - bp.a});
        }
        const size_t sbytes = 16 * dim * ns;
        size_t free_b = 0, total_b = 0;
        CUDA_TRY(c, cudaMemGetInfo(&free_b, &total_b));
        if ((double)sbytes * c->nb > 0.85 * (double)free_b)
            return fail(c, HVP_ENOMEM, fmt("HVP_TENSOR: %d block-boundary state sets of %zu bytes do not fit in 85%% of "
                                          "the free device memory", c->nb, sbytes));
        if ((rc = dalloc(c, (void**)&c->d_blocks, sizeof(DevBlock) * db.size()))) return rc;
        if ((rc = dalloc(c, (void**)&c->d_bgates, sizeof(DevBlockGate) * dbg.size()))) return rc;
        CUDA_TRY(c, cudaMemcpy(c->d_blocks, db.data(), sizeof(DevBlock) * db.size(), cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(c->d_bgates, dbg.data(), sizeof(DevBlockGate) * dbg.size(), cudaMemcpyHostToDevice));
        if ((rc = dalloc(c, (void**)&c->d_mats64, sizeof(Mats64) * (size_t)c->K))) return rc;
        if ((rc = dalloc(c, (void**)&c->d_ops, sizeof(uint32_t) * kOpWords * (size_t)c->nb))) return rc;
        if ((rc = dalloc(c, (void**)&c->d_rec, sizeof(double) * 16384 * (size_t)c->nb * c->tc_ctas_bwd))) return rc;
        if ((rc = dalloc(c, (void**)&c->d_psum, sizeof(double) * 16384 * (size_t)c->nb))) return rc;
        if ((rc = dalloc(c, (void**)&c->d_Ew, sizeof(double2) * 16 * (size_t)c->K))) return rc;
        if ((rc = dalloc(c, (void**)&c->d_DEw, sizeof(double2) * 16 * (size_t)c->K))) return rc;
        if ((rc = dalloc(c, (void**)&c->d_ovl, sizeof(double) * 4 * (size_t)ns * c->ovl_chunks))) return rc;
        c->tstate.assign(c->nb, nullptr);
        for (int j = 0; j < c->nb; ++j)
            if ((rc = dalloc(c, &c->tstate[j], sbytes))) return rc;
        if ((rc = dalloc(c, &c->d_psi0, sbytes))) return rc;
    } else if (c->unfused) {
        if ((rc = dalloc(c, &c->d_x, state_elt(c) * dim * ns))) return rc;
    } else {
        std::vector<DevPass> dp;
        std::vector<DevGate> dg;
        build_dev_passes(c->plan, dp, dg);
        if ((rc = dalloc(c, (void**)&c->d_pass, sizeof(DevPass) * dp.size()))) return rc;
        if ((rc = dalloc(c, (void**)&c->d_gates, sizeof(DevGate) * std::max<size_t>(dg.size(), 1)))) return rc;
        CUDA_TRY(c, cudaMemcpy(c->d_pass, dp.data(), sizeof(DevPass) * dp.size(), cudaMemcpyHostToDevice));
        if (!dg.empty())
            CUDA_TRY(c, cudaMemcpy(c->d_gates, dg.data(), sizeof(DevGate) * dg.size(), cudaMemcpyHostToDevice));
        const int P = c->P;
        const size_t sbytes = state_elt(c) * dim * ns;
        size_t free_b = 0, total_b = 0;
        CUDA_TRY(c, cudaMemGetInfo(&free_b, &total_b));
        // Forward-cache schedule (the states before every gate kept, K slots of
        // one state set each) when the caller did not ask for recomputation or
        // for a checkpoint stride, the scalar kernels are selected, the cached
        // backward pass fits in shared memory and the cache plus the chained
        // boundary states fit in 85 % of the free device memory.
        const size_t slot = (multi ? 24 : 16) * dim * ns;
        const bool cache_fits = !(tuned.flags & HVP_RECOMPUTE) && cfg->checkpoint_stride == 0 && c->variant == 1 &&
                                (c->threads == 128 || c->threads == 256) &&
                                tiled_cached_smem_bytes(true, c->w, c->threads, c->max_gates) <= 227 * 1024 &&
                                (!multi || pair_smem_bytes(true, c->w, 256, c->max_gates) <= 227 * 1024) &&
                                (double)slot * c->K + (multi ? 1.5 : 1.0) * (double)sbytes <= 0.85 * (double)free_b;
        if (cache_fits) {
            if ((rc = dalloc(c, &c->d_cache, slot * (size_t)c->K))) return rc;
            if ((rc = dalloc(c, &c->d_chain, (multi ? 24 : 16) * dim * ns))) return rc;
            c->cache = true;
            c->cache_slot = slot;
            if (multi) {   // second direction's matrices, records and results
                CUDA_TRY(c, pair_set_smem_limits());
                if ((rc = dalloc(c, (void**)&c->d_V2, 16 * 16 * (size_t)c->K))) return rc;
                if ((rc = dalloc(c, &c->d_mats2, sizeof(Mats32) * (size_t)c->K))) return rc;
                if ((rc = dalloc(c, (void**)&c->d_partial2, 64 * sizeof(double) * (size_t)c->K * ns * c->cx_count)))
                    return rc;
                if ((rc = dalloc(c, (void**)&c->d_env2, 64 * sizeof(double) * (size_t)c->K * ns))) return rc;
                if ((rc = dalloc(c, (void**)&c->d_res2, sizeof(double) * c->res_len))) return rc;
                CUDA_TRY(c, cudaMemset(c->d_res2, 0, sizeof(double) * c->res_len));
                CUDA_TRY(c, cudaMallocHost((void**)&c->h_res2, sizeof(double) * c->res_len));
                c->pair = true;
            }
            c->stride = 1;
            c->s0_last = 0;
            c->ckpt.assign(P + 1, nullptr);
        }
        // Checkpoint stride: every boundary if memory allows, else the smallest
        // stride that fits in 85% of the free device memory.
        int cs = cfg->checkpoint_stride;
        auto need = [&](int s) {
            const int stored = (P - 1) / s;
            const int s0_last = ((P - 1) / s) * s;
            const int slots = std::max(s - 1, P - 1 - s0_last);
            const bool scratch = s > 1 && s0_last > 1;
            return sbytes * (size_t)(stored + slots + (scratch ? 1 : 0));
        };
        if (cs == 0) {
            cs = 1;
            while (cs < std::max(P, 1) && need(cs) > (size_t)(0.85 * (double)free_b)) ++cs;
        }
        cs = std::max(1, std::min(cs, std::max(P, 1)));
        if (!c->cache) {
            c->stride = cs;
            c->s0_last = ((P - 1) / cs) * cs;
            c->ckpt.assign(P + 1, nullptr);
            for (int j = 1; j <= P - 1; ++j)
                if (j % cs == 0)
                    if ((rc = dalloc(c, &c->ckpt[j], sbytes))) return rc;
            c->n_slots = std::max(cs - 1, P - 1 - c->s0_last);
            c->slots.assign(c->n_slots, nullptr);
            for (int i = 0; i < c->n_slots; ++i)
                if ((rc = dalloc(c, &c->slots[i], sbytes))) return rc;
            if (cs > 1 && c->s0_last > 1)
                if ((rc = dalloc(c, &c->d_scratch, sbytes))) return rc;
        }
    }

    // Input states.
    double* tmp = nullptr;
    const size_t tmp_bytes = sizeof(double) * std::max((size_t)ns * n * 4, (cfg->flags & HVP_PHI_GIVEN) ? dim * ns * 2 : 0);
    if (c->bytes + tmp_bytes > device_alloc_cap())
        return fail(c, HVP_ENOMEM, "temporary input buffer exceeds the cap HVP_DEVICE_ALLOC_CAP_MB");
    if (cudaMalloc((void**)&tmp, tmp_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, HVP_ENOMEM, "temporary input buffer");
    }
    struct TmpFree { double* p; ~TmpFree() { cudaFree(p); } } tmp_guard{tmp};
    CUDA_TRY(c, cudaMemcpy(tmp, psi_1q, sizeof(double) * ns * n * 4, cudaMemcpyHostToDevice));
    if (c->dbl) CUDA_TRY(c, cudaMemcpy(c->d_psi1q, tmp, sizeof(double) * ns * n * 4, cudaMemcpyDeviceToDevice));
    else CUDA_TRY(c, launch_psi1q_convert(tmp, (float2*)c->d_psi1q, (size_t)ns * n * 2, c->stream));
    if (c->tensor)   // the block passes read the product input states like any other block input
        CUDA_TRY(c, launch_product_states((const float2*)c->d_psi1q, (float4*)c->d_psi0, n, ns, c->stream));
    if (cfg->flags & HVP_PHI_GIVEN) {
        std::vector<int> pos(n);
        if (c->unfused || c->tensor) {
            for (int q = 0; q < n; ++q) pos[q] = n - 1 - q;
        } else {
            pos = c->plan.passes[c->P - 1].pos_in;
        }
        int* dpos = nullptr;
        if ((rc = dalloc(c, (void**)&dpos, sizeof(int) * n))) return rc;
        CUDA_TRY(c, cudaMemcpyAsync(tmp, ref, sizeof(double) * dim * ns * 2, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(dpos, pos.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(c, launch_phi_permute((const double2*)tmp, c->d_phi, c->dbl, n, ns, dpos, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    } else {
        if ((rc = compute_phi_from_uref(c, ref))) return rc;
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    CUDA_TRY(c, cudaGetLastError());
    return HVP_OK;
}

int call_impl(hvp_ctx* c, const double* G, const double* V, double* loss, double* grad, double* hvp_out) {
    if (!c) return HVP_EINVAL;
    if (!G) return fail(c, HVP_EINVAL, "G is NULL");
    if (c->batch) {
        const size_t n32b = 32 * (size_t)c->K;
        if (!all_finite(G, n32b) || (V && !all_finite(V, n32b))) return fail(c, HVP_ENONFINITE, "G or V is not finite");
        std::string e;
        int rc = batch_call(c->batch, G, V, false, loss, grad, hvp_out, e);
        return rc ? fail(c, rc, e) : HVP_OK;
    }
    const size_t n32 = 32 * c->n_user();
    const bool tan = V != nullptr;
    if (!all_finite(G, n32) || (tan && !all_finite(V, n32))) return fail(c, HVP_ENONFINITE, "G or V is not finite");
    std::memcpy(c->h_in, G, sizeof(double) * n32);
    if (tan) std::memcpy(c->h_in + n32, V, sizeof(double) * n32);
    CUDA_TRY(c, cudaMemcpyAsync(c->in_G(), c->h_in, sizeof(double) * n32, cudaMemcpyHostToDevice, c->stream));
    if (tan)
        CUDA_TRY(c, cudaMemcpyAsync(c->in_V(), c->h_in + n32, sizeof(double) * n32, cudaMemcpyHostToDevice, c->stream));
    int rc = run(c, tan);
    if (rc) return rc;
    CUDA_TRY(c, cudaMemcpyAsync(c->h_res, c->d_res, sizeof(double) * c->res_len, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (*c->h_status & 2) return fail(c, HVP_ETIMEOUT, "a bounded wait for a forward-cache copy expired");
    if (*c->h_status) return fail(c, HVP_ENONFINITE, "a gate is singular or not finite");
    const bool riem = (c->cfg.flags & HVP_RIEMANNIAN) != 0;
    const double* g = c->h_res + c->uoff(riem ? 2 : 0);
    const double* h = c->h_res + c->uoff(riem ? 3 : 1);
    if (!all_finite(c->h_res, c->off_ge()) || !all_finite(g, n32) || (tan && !all_finite(h, n32)))
        return fail(c, HVP_ENONFINITE, "non-finite result");
    if (loss) *loss = c->h_res[0];
    if (grad) std::memcpy(grad, g, sizeof(double) * n32);
    if (hvp_out && tan) std::memcpy(hvp_out, h, sizeof(double) * n32);
    return HVP_OK;
}

}  // namespace

int hvp_internal_copy_phi(hvp_ctx* c, void* dst, size_t bytes) {
    if (!c || c->unfused || c->dbl) return HVP_EINVAL;
    if (cudaMemcpyAsync(dst, c->d_phi, bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return HVP_ECUDA;
    return HVP_OK;
}

extern "C" {

int hvp_init(hvp_ctx** out, const hvp_config* cfg, const double* psi_1q, const double* ref_data) {
    NvtxRange range("hvp_init");
    if (!out) return fail(nullptr, HVP_EINVAL, "hvp_init: out is NULL");
    *out = nullptr;
    hvp_ctx* c = new (std::nothrow) hvp_ctx();
    if (!c) return fail(nullptr, HVP_ENOMEM, "out of host memory");
    int rc = init_impl(c, cfg, psi_1q, ref_data);
    if (rc) {
        g_init_error = c->err;
        hvp_free(c);
        return rc;
    }
    *out = c;
    return HVP_OK;
}

int hvp_init_batch(hvp_ctx** out, int n_circuits, const hvp_config* cfgs, const double* const* psi_1q,
                   const double* const* ref_data) {
    NvtxRange range("hvp_init_batch");
    if (!out) return fail(nullptr, HVP_EINVAL, "hvp_init_batch: out is NULL");
    *out = nullptr;
    if (n_circuits < 1 || !cfgs || !psi_1q || !ref_data)
        return fail(nullptr, HVP_EINVAL, "hvp_init_batch: bad arguments");
    for (int c = 0; c < n_circuits; ++c) {
        const hvp_config& f = cfgs[c];
        if (f.n < 2 || f.n > kMaxN || f.n_layers < 1 || f.n_samples < 1 || !psi_1q[c] || !ref_data[c])
            return fail(nullptr, HVP_EINVAL, fmt("hvp_init_batch: circuit %d has a bad shape or NULL input", c));
        if (f.precision != HVP_C64 || (f.flags & HVP_UNFUSED))
            return fail(nullptr, HVP_EINVAL, "hvp_init_batch: batches run the complex64 window-pass path");
        if (f.n > 12 && ((size_t)1 << f.n) * (size_t)f.n_samples > ((size_t)1 << 30))
            return fail(nullptr, HVP_EINVAL, "hvp_init_batch: a circuit above 2^30 amplitudes");
        if (!all_finite(psi_1q[c], (size_t)f.n_samples * f.n * 4)) return fail(nullptr, HVP_ENONFINITE, "psi_1q is not finite");
    }
    if (cfgs[0].window != 0 && (cfgs[0].window < 6 || cfgs[0].window > 12))
        return fail(nullptr, HVP_EINVAL, "hvp_init_batch: window must be 0 or 6..12");
    hvp_ctx* c = new (std::nothrow) hvp_ctx();
    if (!c) return fail(nullptr, HVP_ENOMEM, "out of host memory");
    c->cfg = cfgs[0];
    c->n_circuits = n_circuits;
    for (int i = 0; i < n_circuits; ++i) c->K += num_gates(cfgs[i].n, cfgs[i].n_layers);
    if (cudaSetDevice(cfgs[0].device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return fail(nullptr, HVP_ECUDA, "hvp_init_batch: cudaSetDevice failed");
    }
    if (cfgs[0].stream) {
        c->stream = (cudaStream_t)cfgs[0].stream;
    } else if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) == cudaSuccess) {
        c->own_stream = true;
    } else {
        delete c;
        return fail(nullptr, HVP_ECUDA, "hvp_init_batch: stream creation failed");
    }
    tiled_set_smem_limits();
    std::string e;
    int window = cfgs[0].window > 0 ? cfgs[0].window : 12;
    int max_n = 0;
    for (int i = 0; i < n_circuits; ++i) max_n = std::max(max_n, cfgs[i].n);
    if ((cfgs[0].flags & HVP_AUTOTUNE) && max_n > 12) {
        // Autotuning of the window width of the circuits that run window
        // passes (the number of qubits whose gates are applied per HBM round
        // trip): build the batch for each candidate, time two calls with
        // identity gates (the cost of a sweep does not depend on the gate
        // values) and keep the fastest.
        std::vector<double> eye(32 * (size_t)c->K, 0.0), res(64 * (size_t)c->K + 2 * n_circuits);
        for (int k = 0; k < c->K; ++k)
            for (int d = 0; d < 4; ++d) eye[32 * (size_t)k + 2 * (d * 4 + d)] = 1.0;
        double best = 1e300;
        for (int cand : {12, 11, 10}) {
            BatchImpl* bi = nullptr;
            std::string e2;
            if (batch_init(&bi, n_circuits, cfgs, psi_1q, ref_data, c->stream, cand, e2) != HVP_OK) {
                batch_free(bi);
                continue;
            }
            double* loss = res.data();
            double* g = loss + n_circuits;
            double* h = g + 32 * (size_t)c->K;
            int ok = batch_call(bi, eye.data(), eye.data(), false, loss, g, h, e2);
            auto t0 = std::chrono::steady_clock::now();
            for (int r = 0; r < 2 && ok == HVP_OK; ++r) ok = batch_call(bi, eye.data(), eye.data(), false, loss, g, h, e2);
            const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            batch_free(bi);
            if (ok == HVP_OK && dt < best) {
                best = dt;
                window = cand;
            }
        }
        cudaGetLastError();
    }
    int rc = batch_init(&c->batch, n_circuits, cfgs, psi_1q, ref_data, c->stream, window, e);
    if (rc) {
        c->batch = nullptr;
        g_init_error = e;
        hvp_free(c);
        return rc;
    }
    *out = c;
    return HVP_OK;
}

int hvp_loss_grad(hvp_ctx* ctx, const double* G, double* loss, double* grad) {
    NvtxRange range("hvp_loss_grad");
    return call_impl(ctx, G, nullptr, loss, grad, nullptr);
}

int hvp_hvp(hvp_ctx* ctx, const double* G, const double* V, double* loss, double* grad, double* hvp) {
    NvtxRange range("hvp_hvp");
    if (ctx && !V) return fail(ctx, HVP_EINVAL, "V is NULL");
    return call_impl(ctx, G, V, loss, grad, hvp);
}

int hvp_hvp_dev(hvp_ctx* c, const double* G_dev, const double* V_dev, double* loss_dev, double* grad_dev,
                double* hvp_dev) {
    NvtxRange range("hvp_hvp_dev");
    if (!c) return HVP_EINVAL;
    if (!G_dev) return fail(c, HVP_EINVAL, "G_dev is NULL");
    if (c->batch) {
        std::string e;
        int rcb = batch_call(c->batch, G_dev, V_dev, true, loss_dev, grad_dev, hvp_dev, e);
        return rcb ? fail(c, rcb, e) : HVP_OK;
    }
    const size_t n32 = 32 * c->n_user();
    const bool tan = V_dev != nullptr;
    CUDA_TRY(c, cudaMemcpyAsync(c->in_G(), G_dev, sizeof(double) * n32, cudaMemcpyDeviceToDevice, c->stream));
    if (tan) CUDA_TRY(c, cudaMemcpyAsync(c->in_V(), V_dev, sizeof(double) * n32, cudaMemcpyDeviceToDevice, c->stream));
    int rc = run(c, tan);
    if (rc) return rc;
    const bool riem = (c->cfg.flags & HVP_RIEMANNIAN) != 0;
    if (loss_dev) CUDA_TRY(c, cudaMemcpyAsync(loss_dev, c->d_res, sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    if (grad_dev)
        CUDA_TRY(c, cudaMemcpyAsync(grad_dev, c->d_res + c->uoff(riem ? 2 : 0), sizeof(double) * n32,
                                    cudaMemcpyDeviceToDevice, c->stream));
    if (hvp_dev && tan)
        CUDA_TRY(c, cudaMemcpyAsync(hvp_dev, c->d_res + c->uoff(riem ? 3 : 1), sizeof(double) * n32,
                                    cudaMemcpyDeviceToDevice, c->stream));
    return HVP_OK;
}

int hvp_hvp_multi_dev(hvp_ctx* c, const double* G_dev, int n_dir, const double* V_dev, double* loss_dev,
                      double* grad_dev, double* hvp_dev) {
    NvtxRange range("hvp_hvp_multi_dev");
    if (!c) return HVP_EINVAL;
    if (!G_dev || !V_dev || n_dir < 1) return fail(c, HVP_EINVAL, "hvp_hvp_multi_dev: NULL input or n_dir < 1");
    if (c->batch) return fail(c, HVP_EINVAL, "hvp_hvp_multi_dev: not available for a batch context");
    const size_t n32 = 32 * (size_t)c->K;
    const bool riem = (c->cfg.flags & HVP_RIEMANNIAN) != 0;
    const size_t off_h = riem ? c->off_hr() : c->off_he();
    int d = 0;
    if (c->pair) {
        CUDA_TRY(c, cudaMemcpyAsync(c->d_G, G_dev, sizeof(double) * n32, cudaMemcpyDeviceToDevice, c->stream));
        for (; d + 1 < n_dir; d += 2) {
            CUDA_TRY(c, cudaMemcpyAsync(c->d_V, V_dev + d * n32, sizeof(double) * n32, cudaMemcpyDeviceToDevice,
                                        c->stream));
            CUDA_TRY(c, cudaMemcpyAsync(c->d_V2, V_dev + (d + 1) * n32, sizeof(double) * n32,
                                        cudaMemcpyDeviceToDevice, c->stream));
            int rc = run_pair(c);
            if (rc) return rc;
            if (hvp_dev) {
                CUDA_TRY(c, cudaMemcpyAsync(hvp_dev + d * n32, c->d_res + off_h, sizeof(double) * n32,
                                            cudaMemcpyDeviceToDevice, c->stream));
                CUDA_TRY(c, cudaMemcpyAsync(hvp_dev + (d + 1) * n32, c->d_res2 + off_h, sizeof(double) * n32,
                                            cudaMemcpyDeviceToDevice, c->stream));
            }
            if (d == 0) {
                if (loss_dev)
                    CUDA_TRY(c, cudaMemcpyAsync(loss_dev, c->d_res, sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
                if (grad_dev)
                    CUDA_TRY(c, cudaMemcpyAsync(grad_dev, c->d_res + (riem ? c->off_gr() : c->off_ge()),
                                                sizeof(double) * n32, cudaMemcpyDeviceToDevice, c->stream));
            }
        }
    }
    const size_t nu32 = 32 * c->n_user();
    for (; d < n_dir; ++d) {   // one direction per sweep
        int rc = hvp_hvp_dev(c, G_dev, V_dev + d * nu32, d == 0 ? loss_dev : nullptr, d == 0 ? grad_dev : nullptr,
                             hvp_dev ? hvp_dev + d * nu32 : nullptr);
        if (rc) return rc;
    }
    return HVP_OK;
}

int hvp_hvp_multi(hvp_ctx* c, const double* G, int n_dir, const double* V, double* loss, double* grad,
                  double* hvp) {
    NvtxRange range("hvp_hvp_multi");
    if (!c) return HVP_EINVAL;
    if (!G || !V || n_dir < 1) return fail(c, HVP_EINVAL, "hvp_hvp_multi: NULL input or n_dir < 1");
    if (c->batch) return fail(c, HVP_EINVAL, "hvp_hvp_multi: not available for a batch context");
    const size_t n32 = 32 * c->n_user();
    if (!all_finite(G, n32) || !all_finite(V, n32 * n_dir)) return fail(c, HVP_ENONFINITE, "G or V is not finite");
    const bool riem = (c->cfg.flags & HVP_RIEMANNIAN) != 0;
    int d = 0;
    if (c->pair) {
        std::memcpy(c->h_in, G, sizeof(double) * n32);
        CUDA_TRY(c, cudaMemcpyAsync(c->d_G, c->h_in, sizeof(double) * n32, cudaMemcpyHostToDevice, c->stream));
        for (; d + 1 < n_dir; d += 2) {
            CUDA_TRY(c, cudaStreamSynchronize(c->stream));   // h_in is reused
            std::memcpy(c->h_in + n32, V + d * n32, sizeof(double) * n32);
            CUDA_TRY(c, cudaMemcpyAsync(c->d_V, c->h_in + n32, sizeof(double) * n32, cudaMemcpyHostToDevice,
                                        c->stream));
            CUDA_TRY(c, cudaMemcpyAsync(c->d_V2, V + (d + 1) * n32, sizeof(double) * n32, cudaMemcpyHostToDevice,
                                        c->stream));
            int rc = run_pair(c);
            if (rc) return rc;
            CUDA_TRY(c, cudaMemcpyAsync(c->h_res, c->d_res, sizeof(double) * c->res_len, cudaMemcpyDeviceToHost,
                                        c->stream));
            CUDA_TRY(c, cudaMemcpyAsync(c->h_res2, c->d_res2, sizeof(double) * c->res_len, cudaMemcpyDeviceToHost,
                                        c->stream));
            CUDA_TRY(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(c, cudaStreamSynchronize(c->stream));
            if (*c->h_status & 2) return fail(c, HVP_ETIMEOUT, "a bounded wait for a forward-cache copy expired");
            if (*c->h_status) return fail(c, HVP_ENONFINITE, "a gate is singular or not finite");
            const double* g = c->h_res + (riem ? c->off_gr() : c->off_ge());
            const double* h1 = c->h_res + (riem ? c->off_hr() : c->off_he());
            const double* h2 = c->h_res2 + (riem ? c->off_hr() : c->off_he());
            if (!all_finite(c->h_res, c->off_ge() + n32) || !all_finite(g, n32) || !all_finite(h1, n32) ||
                !all_finite(h2, n32))
                return fail(c, HVP_ENONFINITE, "non-finite result");
            if (d == 0) {
                if (loss) *loss = c->h_res[0];
                if (grad) std::memcpy(grad, g, sizeof(double) * n32);
            }
            if (hvp) {
                std::memcpy(hvp + d * n32, h1, sizeof(double) * n32);
                std::memcpy(hvp + (d + 1) * n32, h2, sizeof(double) * n32);
            }
        }
    }
    for (; d < n_dir; ++d) {
        int rc = call_impl(c, G, V + d * n32, d == 0 ? loss : nullptr, d == 0 ? grad : nullptr,
                           hvp ? hvp + d * n32 : nullptr);
        if (rc) return rc;
    }
    return HVP_OK;
}

int hvp_profile(hvp_ctx* c, const double* G_dev, const double* V_dev, int max_launches, float* ms, int* kind,
                double* flops, double* bytes) {
    NvtxRange range("hvp_profile");
    if (!c || !G_dev || max_launches < 0) return HVP_EINVAL;
    if (c->batch) return fail(c, HVP_EINVAL, "hvp_profile: not available for a batch context");
    const size_t n32 = 32 * c->n_user();
    const bool tan = V_dev != nullptr;
    CUDA_TRY(c, cudaMemcpyAsync(c->in_G(), G_dev, sizeof(double) * n32, cudaMemcpyDeviceToDevice, c->stream));
    if (tan) CUDA_TRY(c, cudaMemcpyAsync(c->in_V(), V_dev, sizeof(double) * n32, cudaMemcpyDeviceToDevice, c->stream));
    cudaEvent_t start;
    CUDA_TRY(c, cudaEventCreate(&start));
    CUDA_TRY(c, cudaEventRecord(start, c->stream));
    c->prof = true;
    int rc = enqueue_all(c, tan);
    c->prof = false;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    int count = (int)c->prof_ev.size();
    if (!rc && e == cudaSuccess) {
        cudaEvent_t prev = start;
        for (int i = 0; i < count; ++i) {
            float t = 0.f;
            cudaEventElapsedTime(&t, prev, c->prof_ev[i]);
            prev = c->prof_ev[i];
            if (i < max_launches) {
                if (ms) ms[i] = t;
                if (kind) kind[i] = c->prof_kind[i];
                if (flops) flops[i] = c->prof_flops[i];
                if (bytes) bytes[i] = c->prof_bytes[i];
            }
        }
    }
    cudaEventDestroy(start);
    for (auto ev : c->prof_ev) cudaEventDestroy(ev);
    c->prof_ev.clear();
    c->prof_kind.clear();
    c->prof_flops.clear();
    c->prof_bytes.clear();
    if (rc) return rc;
    if (e != cudaSuccess) return fail(c, HVP_ECUDA, fmt("profiling run failed: %s", cudaGetErrorString(e)));
    return count;
}

int hvp_get(hvp_ctx* c, int what, double* out) {
    if (!c || !out) return HVP_EINVAL;
    if (c->batch) {
        std::string e;
        int rcb = batch_get(c->batch, what, out, e);
        return rcb ? fail(c, rcb, e) : HVP_OK;
    }
    size_t off = 0, len = 0;
    const size_t n32 = 32 * c->n_user(), ns = c->cfg.n_samples;
    switch (what) {
        case HVP_OUT_T: off = c->off_T(); len = 2 * ns; break;
        case HVP_OUT_OMEGA: off = c->off_Om(); len = 2 * ns; break;
        case HVP_OUT_GRAD_E: off = c->uoff(0); len = n32; break;
        case HVP_OUT_HVP_E: off = c->uoff(1); len = n32; break;
        case HVP_OUT_GRAD_R: off = c->uoff(2); len = n32; break;
        case HVP_OUT_HVP_R: off = c->uoff(3); len = n32; break;
        case HVP_OUT_LOSS: off = 0; len = 1; break;
        case HVP_OUT_ENV:
            if (c->tensor)
                return fail(c, HVP_EINVAL, "HVP_OUT_ENV: the HVP_TENSOR schedule sums environments over samples");
            CUDA_TRY(c, cudaMemcpyAsync(out, c->d_env, sizeof(double) * 64 * c->K * ns, cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(c, cudaStreamSynchronize(c->stream));
            return HVP_OK;
        default: return fail(c, HVP_EINVAL, "unknown output selector");
    }
    CUDA_TRY(c, cudaMemcpyAsync(out, c->d_res + off, sizeof(double) * len, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return HVP_OK;
}

int hvp_plan_info(const hvp_ctx* c, long long info[10]) {
    if (!c || !info) return HVP_EINVAL;
    if (c->batch) {
        batch_info(c->batch, info);
        return HVP_OK;
    }
    info[0] = c->K;
    if (c->tensor) {
        info[1] = c->nb;
        info[2] = kBlockQ;
        info[3] = 0;
        info[4] = c->launches_per_call[1];
        info[5] = (long long)(c->bytes >> 20);
        info[6] = 0;
        info[7] = c->tc_ctas_bwd;
        info[8] = 256;
        info[9] = 0;
        return HVP_OK;
    }
    info[1] = c->unfused ? c->K : c->P;
    info[2] = c->w;
    info[3] = c->cache ? 0 : c->stride;
    info[4] = c->launches_per_call[1];
    info[5] = (long long)(c->bytes >> 20);
    info[6] = c->tiles_per_cta;
    info[7] = c->cx_count;
    info[8] = c->threads;
    info[9] = c->variant;
    return HVP_OK;
}

int hvp_batch_wait_test(hvp_ctx* c, int dep_bias, long long spin_limit) {
    if (!c) return fail(nullptr, HVP_EINVAL, "hvp_batch_wait_test: ctx is NULL");
    if (!c->batch) return fail(c, HVP_EINVAL, "hvp_batch_wait_test: not a batch context");
    if (dep_bias < 0 || dep_bias > 1 || spin_limit < 1)
        return fail(c, HVP_EINVAL, "hvp_batch_wait_test: dep_bias must be 0 or 1 and spin_limit >= 1");
    return batch_wait_test(c->batch, dep_bias, spin_limit);
}

int hvp_cache_wait_test(hvp_ctx* c, int extra_bytes, long long spin_limit) {
    if (!c) return fail(nullptr, HVP_EINVAL, "hvp_cache_wait_test: ctx is NULL");
    if (!c->cache && !c->tensor)
        return fail(c, HVP_EINVAL, "hvp_cache_wait_test: the context does not run the forward cache");
    if ((extra_bytes != 0 && extra_bytes != 16) || spin_limit < 0 || spin_limit > 0x7fffffffll)
        return fail(c, HVP_EINVAL, "hvp_cache_wait_test: extra_bytes must be 0 or 16, spin_limit in [0, 2^31)");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (c->tensor) {
        c->tc_wait_limit = extra_bytes ? (unsigned)std::max<long long>(1, spin_limit) : 0u;
        c->tc_barrier_extra = extra_bytes ? 1u : 0u;
    }
    c->copy_extra_bytes = (unsigned)extra_bytes;
    c->copy_wait_limit = (unsigned)spin_limit;
    for (auto& g : c->gexec)   // the kernel arguments are baked into the captured graphs
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    if (c->gexec_pair) {
        cudaGraphExecDestroy(c->gexec_pair);
        c->gexec_pair = nullptr;
    }
    return HVP_OK;
}

void hvp_free(hvp_ctx* c) {
    if (!c) return;
    if (c->batch) {
        batch_free(c->batch);
        c->batch = nullptr;
    }
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto& g : c->gexec)
        if (g) cudaGraphExecDestroy(g);
    if (c->gexec_pair) cudaGraphExecDestroy(c->gexec_pair);
    if (c->h_res2) cudaFreeHost(c->h_res2);
    for (void* p : c->allocs) cudaFree(p);
    if (c->h_in) cudaFreeHost(c->h_in);
    if (c->h_res) cudaFreeHost(c->h_res);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char* hvp_last_error(const hvp_ctx* c) {
    if (c) return c->err.c_str();
    return g_init_error.c_str();
}

}  // extern "C"
