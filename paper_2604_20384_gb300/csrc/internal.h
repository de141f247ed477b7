// Internal declarations shared by the translation units of libhvp.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cstdlib>

namespace hvp {

// Failure injection on the host: with HVP_DEVICE_ALLOC_CAP_MB set, a context
// (or batch) whose device allocations would exceed that many MiB fails with
// HVP_ENOMEM exactly as if cudaMalloc had failed (tests of the error path).
inline size_t device_alloc_cap() {
    const char* v = std::getenv("HVP_DEVICE_ALLOC_CAP_MB");
    if (!v || !*v) return ~(size_t)0;
    char* end = nullptr;
    const unsigned long long mb = std::strtoull(v, &end, 10);
    if (end == v) return ~(size_t)0;
    return (size_t)mb << 20;
}

constexpr int kMaxN = 30;            // qubits
constexpr int kMaxSamples = 65535;   // samples of one context (grid rows of the window passes)
constexpr int kMaxW = 14;            // local qubits per shared-memory tile
constexpr int kMaxGatesPerPass = 64; // shared-memory budget of one window pass
constexpr int kLowBits = 4;          // address bits every tile keeps contiguous (16 amplitudes)

// ----------------------------------------------------------------- host plan

// One window pass: all gates whose two qubits lie in the window S and whose
// predecessors are done, applied to every tile of 2^|S| amplitudes.
struct PassPlan {
    std::vector<int> S;        // window qubits; shared-memory index bit j <-> qubit S[j]
    std::vector<int> gates;    // gate indices, in an order that respects the circuit
    std::vector<int> pos_in;   // qubit -> amplitude-index bit before the pass
    std::vector<int> pos_out;  // qubit -> amplitude-index bit after the pass
};

struct Plan {
    int n = 0, L = 0, K = 0, w = 0, b = 0;
    std::vector<int> first_qubit;   // gate k acts on (first_qubit[k], first_qubit[k] + 1)
    std::vector<PassPlan> passes;
    std::vector<int> pass_of_gate;
};

// One fused block of the tensor-core schedule: gates acting inside the
// kBlockQ qubits [a, a + kBlockQ), in circuit order.
constexpr int kBlockQ = 5;
struct BlockPlan {
    int a;
    std::vector<int> gates;
};
int make_block_plan(int n, int L, std::vector<BlockPlan>& blocks);

// Device form of a block plan: block j owns the gate records
// [gate_off, gate_off + n_gates) in circuit order.
struct DevBlock {
    int a;          // first qubit of the block
    int n_gates;
    int gate_off;
    int pad;
};
struct DevBlockGate {
    int k;          // gate index
    int u;          // qubit offset of the gate inside the block (0 .. kBlockQ - 2)
};

int num_gates(int n, int L);
void brickwall_layout(int n, int L, std::vector<int>& first_qubit);
// Returns 0 or a negative HVP_* code.
int make_plan(int n, int L, int w, int b, Plan& plan);

// ------------------------------------------------------- device descriptors

// Address and shared-memory index tables of one pass. "Address rank" m
// enumerates the tile's 2^w amplitudes in increasing address order.
struct DevPass {
    int w;                  // local bits of a tile
    int nq;                 // local bits that are qubits (w, or fewer when the
                            // bits above nq select packed samples)
    int ng;                 // global bits (n - w)
    int n_gates;
    int gate_off;           // first entry in the DevGate array
    int gpos[32];           // amplitude-index bit of global tile bit r
    int gq[32];             // qubit at global tile bit r
    int sq[16];             // qubit of shared-memory index bit j
    uint32_t off_lo[64];    // address offset of rank bits [0, 6)
    uint32_t off_hi[256];   // address offset of rank bits [6, w)
    uint16_t in_lo[64], in_hi[256];    // shared-memory index of a rank, input layout
    uint16_t out_lo[64], out_hi[256];  // the same for the output layout
};

struct DevGate {
    int k;   // gate index
    int u;   // shared-memory bit of qubit i (high bit of the 2-bit gate index)
    int v;   // shared-memory bit of qubit i + 1
    int pad;
};

void build_dev_passes(const Plan& plan, std::vector<DevPass>& dp, std::vector<DevGate>& dg);

// ------------------------------------------- fused-block (tensor-core) passes

// One launch applies one block to every amplitude of every sample. Modes:
// forward, X -> [[B, 0], [dB, B]] X; backward, C -> [[B^dag, 0], [dB^dag,
// B^dag]] C with the block environment of the co-states after the update and
// the forward states at the block's input accumulated into rec.
enum TcbMode : int {
    TCB_NO_STORE = 4,    // backward: the updated co-states are not stored (first block)
    TCB_NO_TANGENT = 8,  // the tangent components are zero and stay zero (no GEMM on them)
};

// Operator record of one block (kOpWords 32-bit words). For direction d (0
// forward: B over dB, 1 backward: B^dag over dB^dag), the real 128 x 64
// operator whose rows 2 b' + q (q = re, im) are those of B and rows
// 64 + 2 b' + q those of dB, acting on K = 2 b + (re, im) of 32 block
// amplitudes. Slice i = 0, 1, 2: 128 rows x 32 words, each word two bf16
// integers in [-256, 256] (K element 2w in the low half, 2w + 1 in the high
// half); then the row scales [d][128] as floats. Row m is scale * (s_0 + s_1 /
// 256 + s_2 / 65536) exactly up to 2^-25 of the row's largest entry.
constexpr int kOpSliceWords = 128 * 32;
constexpr int kOpScaleOff = 2 * 3 * kOpSliceWords;
constexpr int kOpWords = kOpScaleOff + 2 * 128;

struct TcbArgs {
    const uint32_t* ops;     // this block's operator record (kOpWords words)
    const float4* xin;       // forward: states at the block's input; backward: co-states
    float4* xout;            // forward: states at the block's output; backward: co-states (in place)
    const float4* psi;       // backward: forward states at the block's input
    double* rec;             // backward: FP64 environment records of this block, [CTA][128][128]
    int* status;             // bit 2: a bounded wait gave up
    long long ncols;         // N_s * 2^(n - 5)
    int n, a, mode;
    unsigned wait_limit;     // polls before a wait gives up (0: the default)
    unsigned barrier_extra;  // test of the bounded waits: arrivals the tile barriers expect beyond the
                             // MMAs' commit (0 in normal use)
    // Tensor maps of xin and psi for the TMA tile loads, and whether each is
    // used (written by launch_tcb from the fields above; without a map the
    // threads load their elements directly).
    int tma_x, tma_p;
    CUtensorMap tm_x;
    CUtensorMap tm_p;
};
cudaError_t launch_tcb(const TcbArgs& a, bool bwd, int ctas, cudaStream_t st);
cudaError_t tcb_set_smem_limits();
int tcb_tiles(long long ncols, bool bwd);
cudaError_t launch_block_prep(const DevBlock* blocks, const DevBlockGate* bg, int nb, const double2* G,
                              const double2* V, uint32_t* ops, int* status, cudaStream_t st);
cudaError_t launch_overlaps(const float4* x, const float2* phi, double* partial, double2* T, double2* Om, int n,
                            int ns, int chunks, cudaStream_t st);
cudaError_t launch_extract_psi(const float4* x, float2* out, size_t count, cudaStream_t st);
cudaError_t launch_product_states(const float2* psi1q, float4* out, int n, int ns, cudaStream_t st);
cudaError_t launch_weighted_phi(const float2* phi, const double2* w1, const double2* w2, float4* out, int n, int ns,
                                cudaStream_t st);

// Swizzle of shared-memory element indices (16-byte elements): conflict-free
// 128-bit accesses when no two neighbouring qubits sit on index bits 0..2.
__host__ __device__ inline unsigned swz(unsigned l) {
    return l ^ ((((l >> 3) ^ (l >> 4)) & 1u) * 7u);
}

// ----------------------------------------------------------- kernel arguments

enum PassMode : int {
    M_GEN = 1,        // generate the product state psi^[0] instead of loading
    M_FWD = 2,        // apply the pass's gates forward
    M_STORE_F = 4,    // store the forward states
    M_BWD = 8,        // apply the pass's gates backward with environment sums
    M_LOAD_PHI = 16,  // co-states start as (phi, 0)
    M_STORE_B = 32,   // store the co-states
};

// Per-gate matrices prepared in FP64 each call: G, G^-1, G^dag, V, V^dag and
// Y = G^-1 V G^-1 (so that dpsi^[k-1] = G^-1 dpsi^[k] - Y psi^[k]).
struct Mats32 { float2 G[16], Ginv[16], Gh[16], V[16], Vh[16], Y[16]; };
struct Mats64 { double2 G[16], Ginv[16], Gh[16], V[16], Vh[16], Y[16]; };
cudaError_t launch_block_post(const DevBlock* blocks, const DevBlockGate* bg, int nb, const double* rec, int cx,
                              double* psum, const Mats64* mats, double2* Ew, double2* DEw, int tangent,
                              cudaStream_t st);

struct TiledArgs {
    const DevPass* pass;
    const DevGate* gates;        // all gates of all passes
    const Mats32* mats;          // K entries
    const float2* psi1q;         // N_s x n x 2
    const void* xin;             // forward states in (float4 or float2 per amplitude)
    void* xout;                  // forward states out
    const float2* phi;           // reference states
    const void* cin;             // co-states in
    void* cout;                  // co-states out
    double* partial;             // [K][N_s][CX][64]
    void* cache;                 // forward cache: slot k = states before gate k (pass order), per
                                 // (sample, tile) one block of 2^w elements in shared-memory order
    size_t cache_slot_bytes;     // bytes of one cache slot (2^n * N_s elements)
    int* status;                 // bit 2: a bounded wait for a cache copy gave up
    const Mats32* mats2;         // second direction's matrices (two-direction passes)
    double* partial2;            // second direction's records (two-direction passes)
    unsigned copy_wait_limit;    // polls before a cache-copy wait gives up (0: the default)
    unsigned copy_extra_bytes;   // test of the bounded waits: bytes the copy barriers expect
                                 // beyond what arrives (0 in normal use)
    int n, n_samples, mode, tiles_per_cta, cx_count;
    int ld_out_tab;              // 1: load through the output-layout tables
    int st_out_tab;              // 1: store through the output-layout tables
};

// Launchers (return cudaError_t of the launch).
// variant 1: scalar FP32 FMAs; 2: packed fma.rn.f32x2; 3: scalar, two groups
// per iteration in the backward kernel. threads: 256 or 512.
cudaError_t launch_tiled(const TiledArgs& a, bool tangent, int w, int threads, int max_gates,
                         cudaStream_t st, int variant = 1);
size_t tiled_smem_bytes(bool tangent, int mode, int w, int threads, int max_gates, int variant = 1);
// Forward-cache schedule: forward passes (mode M_FWD) that also write the
// states before every gate to a.cache, and backward passes (mode M_BWD) that
// read them back instead of recomputing them. threads: 128 or 256.
cudaError_t launch_tiled_cached(const TiledArgs& a, bool tangent, int w, int threads, int max_gates,
                                cudaStream_t st);
size_t tiled_cached_smem_bytes(bool tangent, int w, int threads, int max_gates);
cudaError_t tiled_set_smem_limits();
// Two tangent directions per sweep in the forward-cache schedule (pair.cu):
// forward passes (mode M_FWD) writing a cache of (psi, dpsi_1, dpsi_2), 24
// bytes per amplitude per gate, and backward passes (mode M_BWD) reading it;
// 256 threads.
cudaError_t launch_pair(const TiledArgs& a, int w, int max_gates, cudaStream_t st);
size_t pair_smem_bytes(bool bwd, int w, int threads, int max_gates);
cudaError_t pair_set_smem_limits();

// Unfused (one launch per gate) kernels, real type R = float or double.
cudaError_t unfused_init(bool dbl, const void* psi1q, void* x, int n, int ns, bool tangent, cudaStream_t st);
cudaError_t unfused_fwd_gate(bool dbl, const void* mats, int k, int q, void* x, int n, int ns,
                             bool tangent, cudaStream_t st);
cudaError_t unfused_load_phi(bool dbl, const void* phi, void* c, int n, int ns, bool tangent, cudaStream_t st);
cudaError_t unfused_bwd_gate(bool dbl, const void* mats, int k, int q, void* x, void* c, double* partial,
                             int n, int ns, int cx_count, bool tangent, cudaStream_t st);
int unfused_cx_count(int n, int ns);

// Post-processing (FP64).
struct PostArgs {
    const double* partial;  // [K][N_s][CX][64]
    double* env;            // [N_s][K][64]
    const double2* G;       // K x 16
    const double2* V;       // K x 16 (may be null)
    double2* T;             // N_s
    double2* Omega;         // N_s
    double* loss;           // 1
    double2* grad_e;        // K x 16
    double2* hvp_e;
    double2* grad_r;
    double2* hvp_r;
    int K, n_samples, cx_count, tangent;
    int frobenius;          // 1: derivatives of C_F = 1 - mean Re T instead of C
};
cudaError_t launch_post(const PostArgs& p, cudaStream_t st);
// App. E on the device: layer gates to every gate of the layer, and per-gate
// derivative blocks (four K x 16 outputs, contiguous) to per-layer sums.
cudaError_t launch_expand_layers(const double2* GL, const double2* VL, double2* G, double2* V, const int* first, int L,
                                 cudaStream_t st);
cudaError_t launch_contract_layers(const double2* per_gate, double2* per_layer, const int* first, int L, int K,
                                   cudaStream_t st);
// grad / HVP (Euclidean and App. F) and the loss from sample-summed weighted
// environments (fused-block schedule).
cudaError_t launch_post_weighted(const double2* Ew, const double2* DEw, const double2* G, const double2* V,
                                 const double2* T, double2* ge, double2* he, double2* gr, double2* hr, double* loss,
                                 int K, int ns, int tangent, int frob, cudaStream_t st);
cudaError_t launch_prep(const double2* G, const double2* V, void* mats, bool dbl, int K, int* status,
                        cudaStream_t st);
cudaError_t launch_psi1q_convert(const double* in, float2* out, size_t count, cudaStream_t st);
cudaError_t launch_phi_permute(const double2* phi_std, void* phi_out, bool dbl, int n, int ns,
                               const int* pos, cudaStream_t st);
cudaError_t launch_copy_out(const double* loss, const double2* grad, const double2* hvp,
                            double* loss_dst, double* grad_dst, double* hvp_dst, int K,
                            cudaStream_t st);

void set_thread_error(const char* msg);

// Batched evaluation of many circuits (batch.cu).
struct BatchImpl;


}  // namespace hvp

#include <string>
#include "../../include/hvp.h"

namespace hvp {
int batch_init(BatchImpl** out, int n_circuits, const hvp_config* cfgs, const double* const* psi_1q,
               const double* const* ref, cudaStream_t stream, int window, std::string& err);
int batch_call(BatchImpl* b, const double* G, const double* V, bool dev, double* loss, double* grad, double* hvp,
               std::string& err);
int batch_get(BatchImpl* b, int what, double* out, std::string& err);
void batch_info(const BatchImpl* b, long long* info);
void batch_free(BatchImpl* b);
int batch_wait_test(BatchImpl* b, int dep_bias, long long spin_limit);
}  // namespace hvp

// Copies a context's reference states (FP32, layout of its last pass) to dst.
int hvp_internal_copy_phi(hvp_ctx* ctx, void* dst, size_t bytes);
