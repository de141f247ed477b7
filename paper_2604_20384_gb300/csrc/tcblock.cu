// Tensor-core passes of the fused-block schedule (sm_103a: tcgen05, TMEM).
//
// A pass applies one block of five neighbouring qubits (up to ~10 gates fused
// into a dense 32 x 32 complex operator, App. D's [[B, 0], [dB, B]] for the
// tangent pair) to every amplitude of every sample. Amplitudes are grouped
// into tiles of 32 block amplitudes x 32 "columns" (the other n - 5 qubits and
// the sample); with the four real components (re, im of the state and of its
// tangent) interleaved as 4 b + p, a tile is a real 128 x 32 matrix X and the
// pass is one real GEMM D = A X with the 128 x 128 operator A.
//
// Exact-integer split. The tensor cores' FP32 accumulation truncates, and a
// truncation per accumulation step biases every block application towards
// smaller magnitudes; over the tens of blocks of a sweep that bias exceeds the
// error budget. So each operand is split into three slices of 8-bit integers
// on a power-of-two scale (per row of A, per column and per component group
// of X: the state's two and the tangent's two components carry separate
// scales), x = scale * (s_0 + s_1 / 256 + s_2 / 65536) to 2^-25 of the scale;
// the products of slices and their sums over a K of 64 are integers below
// 2^24, which the bf16 MMAs (kind::f16, FP32 accumulation) produce exactly.
// The GEMM runs as two halves (K = the 64 state components, K = the 64
// tangent components), each with three levels of slice products (i + j = 0,
// 1, 2) in separate TMEM accumulators; the epilogue combines them with
// round-to-nearest FP32 arithmetic:
//     D = rs_0 * cs_psi * (L_00 + L_01 / 256 + L_02 / 65536)
//       + rs_1 * cs_dpsi * (L_10 + L_11 / 256 + L_12 / 65536).
// A (the six operator slices, bf16 pairs) sits in TMEM for the whole launch
// (the A operand of tcgen05.mma may come from TMEM); the slices of X are
// staged in shared memory as K-major operands, two stages deep so that the
// next tile is sliced while the tensor cores work on this one.
//
// Forward: X = (psi, dpsi) at the block's input, D the states at its output.
// Backward: X = the co-states (c, dc) at the block's output, D = [[B^dag, 0],
// [dB^dag, B^dag]] X the co-states at its input (Eq. bis, Eq. dbis); the
// block environment P = D Psi^T (co-states and forward states at the block's
// input, contracted over the tile's columns) is a second GEMM whose A operand
// is D, rewritten in TMEM as TF32 high and low parts, and whose B operand is
// the forward-state tile Psi (three TF32 products). Its per-tile results are
// added to per-thread FP32 sums (round to nearest) and flushed into the CTA's
// FP64 record every 16 tiles, so the truncating accumulation spans one tile.
//
// One CTA per SM (256 threads, all 512 TMEM columns), looping over tiles; one
// thread issues the MMAs and commits them to an mbarrier. Every wait on an
// mbarrier is bounded: a wait that gives up sets bit 2 of *status, the CTA
// leaves its loop together, commits its MMAs in flight to a separate barrier
// and waits (bounded) for it, then frees its TMEM.
#include "internal.h"

namespace hvp {

namespace {

constexpr int kT = 256;                      // threads per CTA
constexpr int TN = 32;                       // columns per tile
constexpr unsigned kTmemCols = 512;
constexpr unsigned kOpCol = 0;               // operator slices (half, slice): 6 x 32 columns
constexpr unsigned kAccCol = 192;            // accumulators (half, level): 6 x 32 columns
constexpr unsigned kEnvCol = 384;            // backward: environment accumulator (128 columns)
constexpr int kFlushTiles = 16;              // FP32 tiles summed before an FP64 flush
constexpr unsigned kWaitLimit = 1u << 22;    // mbarrier polls before a wait gives up

// Shared-memory regions (bytes): X slices (six per stage, K = 64 x 32
// columns, bf16, with the strides below) and, backward, the forward-state
// tile (TF32 high and low, K = 32 columns x 128 rows).
constexpr unsigned kXRegion = 4608;
constexpr unsigned kERegion = 16640;
constexpr unsigned kStageFwd = 6 * kXRegion;
constexpr unsigned kStageBwd = 6 * kXRegion + 2 * kERegion;
constexpr unsigned kStagingBytes = TN * 32 * 16;
constexpr unsigned kCtlBytes = 2 * 2 * 2 * 32 * 4 + 128;  // per stage: column maxima and scales; barriers
constexpr unsigned smem_bytes(bool bwd) {
    return 2 * (bwd ? kStageBwd : kStageFwd) + kStagingBytes + kCtlBytes;
}
// Dynamic shared memory of a launch: at least 116 KB, so that one CTA runs
// per SM (it holds all of the SM's TMEM).
constexpr unsigned launch_smem(bool bwd) { return smem_bytes(bwd) > 116u * 1024u ? smem_bytes(bwd) : 116u * 1024u; }

// Strides of the staged operands (bytes). X slices: K-cores (4 block indices
// x re, im) 144 bytes apart, so that a warp's 4-byte stores of 32 block
// indices of one column hit 32 banks; column cores 1152 apart. Psi tile:
// K-cores (4 columns) 128 apart, row cores 1040 apart (65 16-byte units, so
// that eight lanes' 16-byte stores land in eight bank groups).
constexpr unsigned kLboX = 144, kSboX = 1152, kLboE = 128, kSboE = 1040;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// kind::tf32, FP32 accumulator, both operands K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_tf32(int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_ts(unsigned d, unsigned a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n"
                 :: "r"(d), "r"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned par) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(par)
        : "memory");
    return ok != 0;
}


// Global amplitude index of block index b and column c: c = (sample, the
// other n - 5 qubits in address order); the block's bits are [bl, bl + 5).
__device__ __forceinline__ size_t amp_index(long long c, unsigned b, int n, int bl) {
    const int nr = n - 5;
    const long long s = c >> nr;
    const unsigned long long r = (unsigned long long)c & ((1ull << nr) - 1ull);
    const unsigned long long lo = r & ((1ull << bl) - 1ull), hi = r >> bl;
    return ((size_t)s << n) | (size_t)((hi << (bl + 5)) | ((unsigned long long)b << bl) | lo);
}

// Product state psi^[0] = (x)_q psi_{s,q} at one amplitude (Eq. costHS).
__device__ __forceinline__ float2 product_amp(const float2* __restrict__ q1, size_t g, int n) {
    const size_t s = g >> n;
    const unsigned long long idx = g & ((1ull << n) - 1ull);
    const float2* f = q1 + s * (size_t)n * 2;
    float2 a = make_float2(1.f, 0.f);
    for (int q = 0; q < n; ++q) {
        const float2 v = __ldg(&f[2 * q + ((idx >> (n - 1 - q)) & 1ull)]);
        a = make_float2(a.x * v.x - a.y * v.y, a.x * v.y + a.y * v.x);
    }
    return a;
}


__host__ __device__ constexpr uint32_t idesc_bf16(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma_ts_f16(unsigned d, unsigned a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n"
                 :: "r"(d), "r"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_st16(unsigned taddr, const float (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
        :: "r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
           "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
           "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
           "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
           "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
           "r"(__float_as_uint(v[15]))
        : "memory");
}
__device__ __forceinline__ void tmem_st32u(unsigned taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
        :: "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
           "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]),
           "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]),
           "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

// Power-of-two scale exponent of a column group: 2^e > m >= 2^(e-1) for the
// largest magnitude m (bits of a non-negative float); bounded below so that
// the up-scale 2^(8-e) stays a normal float.
__device__ __forceinline__ int col_exp(unsigned mbits) {
    if (mbits == 0u) return -100;
    const int e = (int)((mbits >> 23) & 255u) - 126;
    return e < -100 ? -100 : e;
}
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((unsigned)(k + 127) << 23); }

// Three 8-bit integer slices of y (|y| < 256): y = s0 + s1 / 256 + s2 / 65536
// up to 2^-17; each slice returned as bf16 bits (exact).
__device__ __forceinline__ void slice3(float y, uint32_t& b0, uint32_t& b1, uint32_t& b2) {
    const float s0 = rintf(y);
    const float r1 = (y - s0) * 256.f;
    const float s1 = rintf(r1);
    const float s2 = rintf((r1 - s1) * 256.f);
    b0 = __float_as_uint(s0) >> 16;
    b1 = __float_as_uint(s1) >> 16;
    b2 = __float_as_uint(s2) >> 16;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Barrier of the 256 worker threads (the MMA warp does not take part).
__device__ __forceinline__ void workers_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Barriers in shared memory (mbarriers):
enum : int {
    B_FULL0 = 0,    // stage 0 staged (256 worker arrivals)
    B_FULL1 = 1,    // stage 1 staged
    B_DONE_U = 2,   // the tile's update MMAs complete (commit)
    B_ACCFREE = 3,  // the workers have read the update accumulators (256 arrivals)
    B_CREADY = 4,   // backward: the co-states are in TMEM as TF32 parts (256 arrivals)
    B_DONE_E = 5,   // backward: the environment MMAs complete (commit)
    B_DRAIN = 6,    // every MMA issued so far complete (commit, on the way out after a failed wait)
    B_COUNT = 7
};

// Warp roles: warps 0-7 (256 threads) load, slice and stage the tiles, read
// the accumulators and store results; warp 8 owns TMEM and its first lane
// issues every MMA, so slicing the next tile overlaps this tile's MMAs.
template <bool BWD>
__global__ void __launch_bounds__(kT + 32, 1) tcb_kernel(TcbArgs a) {
    constexpr unsigned kStage = BWD ? kStageBwd : kStageFwd;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* stagebuf = smem;                                   // [2][kStage]
    float* staging = reinterpret_cast<float*>(smem + 2 * kStage);     // epilogue output tile
    float* csc = reinterpret_cast<float*>(smem + 2 * kStage + kStagingBytes);          // [stage][group][32]
    uint64_t* bars = reinterpret_cast<uint64_t*>(csc + 2 * 2 * 32);                    // [B_COUNT]
    volatile unsigned* ctl = reinterpret_cast<volatile unsigned*>(bars + B_COUNT);    // [tmem base, stop]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool mma_warp = warp == 8;
    const int n = a.n, bl = n - a.a - 5;
    const long long ncols = a.ncols;
    const long long ntiles = (ncols + TN - 1) / TN;
    const unsigned limit = a.wait_limit ? a.wait_limit : kWaitLimit;
    const bool tangent = !(a.mode & TCB_NO_TANGENT);
    const int nh = tangent ? 2 : 1;
    const int dir = BWD ? 1 : 0;

    if (mma_warp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void*)ctl)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        const unsigned extra = a.barrier_extra;
        const unsigned counts[B_COUNT] = {256u, 256u, 1u + extra, 256u, 256u, 1u + extra, 1u};
        for (int i = 0; i < B_COUNT; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars[i])), "r"(counts[i]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        ctl[1] = 0u;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tb = ctl[0];
    const unsigned lane_base = (unsigned)((warp & 3) * 32) << 16;
    const int row = (warp & 3) * 32 + lane;       // TMEM lane = output row 4 b' + p' (worker warps)

    // Operator slices into TMEM: warps 0-3 the three slices of half 0, warps
    // 4-7 those of half 1; each thread its row (32 words = 64 bf16 per slice).
    if (!mma_warp) {
        const int h = warp >> 2;
        for (int i = 0; i < 3; ++i) {
            const uint32_t* src = a.ops + ((dir * 2 + h) * 3 + i) * kOpSliceWords + row * 32;
            uint32_t v[32];
#pragma unroll
            for (int w = 0; w < 32; ++w) v[w] = __ldg(&src[w]);
            tmem_st32u(tb + lane_base + kOpCol + (h * 3 + i) * 32, v);
        }
        tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    // A wait that gives up raises the stop flag; every later wait sees it and
    // returns at once, so all roles leave their loops.
    auto wait = [&](int b, unsigned par) -> bool {
        if (ctl[1]) return false;
        for (unsigned i = 0; i < limit; ++i) {
            if (mbar_try(&bars[b], par)) return true;
            if ((i & 255u) == 255u && ctl[1]) return false;
        }
        ctl[1] = 1u;
        atomicOr(a.status, 2);
        return false;
    };

    if (mma_warp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t id_u = idesc_bf16(TN), id_e = idesc_tf32(128);
            const unsigned sbase = smem_u32(stagebuf);
            const uint64_t kstep_x = (uint64_t)((2u * kLboX) >> 4);
            const uint64_t kstep_e = (uint64_t)((2u * kLboE) >> 4);
            bool issued = false;
            long long i = 0;
            for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
                const int sg = (int)(i & 1);
                if (!wait(B_FULL0 + sg, (unsigned)((i >> 1) & 1))) break;
                if (i > 0) {
                    if (!wait(B_ACCFREE, (unsigned)((i - 1) & 1))) break;
                    if (BWD && !wait(B_DONE_E, (unsigned)((i - 1) & 1))) break;
                }
                tc_fence_after();
                // D = A X: per half, levels 0..2 of slice products (i + j = level), 4 K-steps of 16.
                const unsigned xs = sbase + sg * kStage;
                for (int h = 0; h < nh; ++h)
#pragma unroll
                    for (int lev = 0; lev < 3; ++lev) {
                        const unsigned d = tb + kAccCol + (h * 3 + lev) * 32;
#pragma unroll
                        for (int ii = 0; ii <= lev; ++ii) {
                            const uint64_t bd = sdesc(xs + (h * 3 + lev - ii) * kXRegion, kLboX, kSboX);
                            const unsigned ad = tb + kOpCol + (h * 3 + ii) * 32;
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                mma_ts_f16(d, ad + 8 * k, bd + k * kstep_x, id_u, (ii | k) != 0);
                        }
                    }
                mma_commit(&bars[B_DONE_U]);
                issued = true;
                if constexpr (BWD) {
                    if (!wait(B_CREADY, (unsigned)(i & 1))) break;
                    tc_fence_after();
                    // P = D Psi^T: K = the tile's 32 columns, 4 K-steps; A = D (high, low) from TMEM.
                    const unsigned eb = sbase + sg * kStage + 6 * kXRegion;
                    const uint64_t ph = sdesc(eb, kLboE, kSboE), pl = sdesc(eb + kERegion, kLboE, kSboE);
#pragma unroll
                    for (int k = 0; k < TN / 8; ++k) {
                        mma_ts(tb + kEnvCol, tb + kAccCol + 8 * k, ph + k * kstep_e, id_e, k > 0);
                        mma_ts(tb + kEnvCol, tb + kAccCol + 8 * k, pl + k * kstep_e, id_e, 1);
                        mma_ts(tb + kEnvCol, tb + kAccCol + 32 + 8 * k, ph + k * kstep_e, id_e, 1);
                    }
                    mma_commit(&bars[B_DONE_E]);
                }
            }
            if (ctl[1] && issued) {   // let every MMA issued so far finish (bounded) before TMEM is freed
                mma_commit(&bars[B_DRAIN]);
                for (unsigned k = 0; k < kWaitLimit; ++k)
                    if (mbar_try(&bars[B_DRAIN], 0u)) break;
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ workers
        // Warp w owns the tile's column quad w (columns 4w .. 4w + 3), lane l
        // the block index b = l: a lane loads four columns of one block
        // amplitude (full 32-byte sectors at every block position), and the
        // column maxima are warp reductions.
        const unsigned ub = (unsigned)lane;
        const int uq = warp;
        float4 xr[4], yr[BWD ? 4 : 1];
        float up[2][4];   // per column and component group: 2^(8 - e), e the column's scale exponent
        auto prefetch = [&](long long tile) {
            const long long c0 = tile * TN;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const long long c = c0 + 4 * uq + i;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f), y = v;
                if (c < ncols) {
                    const size_t g = amp_index(c, ub, n, bl);
                    if (!BWD) {
                        if (a.mode & TCB_GEN) {
                            const float2 p = product_amp(a.psi1q, g, n);
                            v = make_float4(p.x, p.y, 0.f, 0.f);
                        } else {
                            v = __ldcs(&a.xin[g]);
                        }
                    } else {
                        if (a.mode & TCB_LOAD_PHI) {
                            const float2 ph = __ldg(&a.phi[g]);
                            const size_t s = g >> n;
                            float2 w1 = make_float2(1.f, 0.f), w2 = make_float2(0.f, 0.f);
                            if (a.w1) w1 = make_float2((float)a.w1[s].x, (float)a.w1[s].y);
                            if (a.w2) w2 = make_float2((float)a.w2[s].x, (float)a.w2[s].y);
                            v = make_float4(w1.x * ph.x - w1.y * ph.y, w1.x * ph.y + w1.y * ph.x,
                                            w2.x * ph.x - w2.y * ph.y, w2.x * ph.y + w2.y * ph.x);
                        } else {
                            v = __ldcs(&a.xin[g]);
                        }
                        if (a.mode & TCB_GEN) {
                            const float2 p = product_amp(a.psi1q, g, n);
                            y = make_float4(p.x, p.y, 0.f, 0.f);
                        } else {
                            y = __ldcs(&a.psi[g]);
                        }
                    }
                    if (!tangent) { v.z = 0.f; v.w = 0.f; y.z = 0.f; y.w = 0.f; }
                }
                xr[i] = v;
                if constexpr (BWD) yr[i] = y;
            }
        };
        // Scale exponents of this warp's four columns (two component groups
        // each): warp-wide maxima; lane 0 publishes the epilogue's scales.
        auto colscale = [&](int sg) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const unsigned m0 = __reduce_max_sync(0xffffffffu, __float_as_uint(fmaxf(fabsf(xr[i].x), fabsf(xr[i].y))));
                const unsigned m1 = __reduce_max_sync(0xffffffffu, __float_as_uint(fmaxf(fabsf(xr[i].z), fabsf(xr[i].w))));
                const int e0 = col_exp(m0), e1 = col_exp(m1);
                up[0][i] = pow2f(8 - e0);
                up[1][i] = pow2f(8 - e1);
                if (lane == 0) {
                    csc[sg * 64 + 4 * uq + i] = pow2f(e0 - 8);
                    csc[sg * 64 + 32 + 4 * uq + i] = pow2f(e1 - 8);
                }
            }
        };
        // Registers -> the slices of stage sg.
        auto stage = [&](int sg) {
            unsigned char* xb = stagebuf + sg * kStage;
            unsigned char* eb = xb + 6 * kXRegion;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int col = 4 * uq + i;
                const unsigned off = (unsigned)(col & 7) * 16u + (ub & 3u) * 4u + (ub >> 2) * kLboX +
                                     (unsigned)(col >> 3) * kSboX;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (h == 1 && !tangent) break;
                    const float re = (h ? xr[i].z : xr[i].x) * up[h][i], im = (h ? xr[i].w : xr[i].y) * up[h][i];
                    uint32_t r0, r1, r2, i0, i1, i2;
                    slice3(re, r0, r1, r2);
                    slice3(im, i0, i1, i2);
                    *reinterpret_cast<uint32_t*>(xb + (h * 3 + 0) * kXRegion + off) = r0 | (i0 << 16);
                    *reinterpret_cast<uint32_t*>(xb + (h * 3 + 1) * kXRegion + off) = r1 | (i1 << 16);
                    *reinterpret_cast<uint32_t*>(xb + (h * 3 + 2) * kXRegion + off) = r2 | (i2 << 16);
                }
            }
            if constexpr (BWD) {
                float4 hi[4], lo[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    hi[i] = make_float4(tf32_rna(yr[i].x), tf32_rna(yr[i].y), tf32_rna(yr[i].z), tf32_rna(yr[i].w));
                    lo[i] = make_float4(tf32_rna(yr[i].x - hi[i].x), tf32_rna(yr[i].y - hi[i].y),
                                        tf32_rna(yr[i].z - hi[i].z), tf32_rna(yr[i].w - hi[i].w));
                }
                // Psi: rows 4 b + p, K = the tile's columns (4 per 16-byte row)
                const unsigned base = (unsigned)uq * kLboE + (ub >> 1) * kSboE + (ub & 1u) * 64u;
                unsigned char* eh = eb;
                unsigned char* el = eb + kERegion;
                *reinterpret_cast<float4*>(eh + base + 0) = make_float4(hi[0].x, hi[1].x, hi[2].x, hi[3].x);
                *reinterpret_cast<float4*>(eh + base + 16) = make_float4(hi[0].y, hi[1].y, hi[2].y, hi[3].y);
                *reinterpret_cast<float4*>(eh + base + 32) = make_float4(hi[0].z, hi[1].z, hi[2].z, hi[3].z);
                *reinterpret_cast<float4*>(eh + base + 48) = make_float4(hi[0].w, hi[1].w, hi[2].w, hi[3].w);
                *reinterpret_cast<float4*>(el + base + 0) = make_float4(lo[0].x, lo[1].x, lo[2].x, lo[3].x);
                *reinterpret_cast<float4*>(el + base + 16) = make_float4(lo[0].y, lo[1].y, lo[2].y, lo[3].y);
                *reinterpret_cast<float4*>(el + base + 32) = make_float4(lo[0].z, lo[1].z, lo[2].z, lo[3].z);
                *reinterpret_cast<float4*>(el + base + 48) = make_float4(lo[0].w, lo[1].w, lo[2].w, lo[3].w);
            }
            fence_async_smem();
        };
        // one tile into stage sg: loads, column scales, slices; then the stage is announced
        auto produce = [&](long long tile, int sg) {
            prefetch(tile);
            colscale(sg);
            stage(sg);
            mbar_arrive(&bars[B_FULL0 + sg]);
        };

        const float* rsc = reinterpret_cast<const float*>(a.ops + kOpScaleOff) + dir * 256;
        const float rs0 = __ldg(&rsc[row]), rs1 = __ldg(&rsc[128 + row]);
        float acc[BWD ? 64 : 1];
#pragma unroll
        for (int i = 0; i < (BWD ? 64 : 1); ++i) acc[i] = 0.f;
        int since_flush = 0;
        bool flushed = false;
        auto flush = [&]() {
            if constexpr (BWD) {
                double* dst = a.rec + (size_t)blockIdx.x * 16384 + (size_t)row * 128 + 64 * (warp >> 2);
#pragma unroll
                for (int i = 0; i < 64; i += 2) {
                    double2 o = make_double2(0.0, 0.0);
                    if (flushed) o = *reinterpret_cast<double2*>(dst + i);
                    o.x += (double)acc[i];
                    o.y += (double)acc[i + 1];
                    *reinterpret_cast<double2*>(dst + i) = o;
                    acc[i] = 0.f;
                    acc[i + 1] = 0.f;
                }
                flushed = true;
                since_flush = 0;
            }
        };

        long long i = 0;
        bool ok = true;
        if ((long long)blockIdx.x < ntiles) produce(blockIdx.x, 0);
        for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
            const int sg = (int)(i & 1);
            const long long next = tile + gridDim.x;
            // the next tile into the other stage, while the MMAs of this one run
            if (next < ntiles) produce(next, sg ^ 1);
            // every worker waits; then all leave together if any wait gave up
            wait(B_DONE_U, (unsigned)(i & 1));
            workers_sync();
            if (ctl[1]) { ok = false; break; }
            tc_fence_after();

            // Epilogue: combine the levels; D -> staging (and, backward, TMEM as TF32 high / low parts).
            const int cc = (warp >> 2) * 16;   // this thread's 16 columns
            const unsigned bb = (unsigned)row >> 2, p = (unsigned)row & 3u;
            float v[16];
            {
                float l0[16], l1[16], l2[16];
                tmem_ld16(tb + lane_base + kAccCol + 0 * 32 + cc, l0);
                tmem_ld16(tb + lane_base + kAccCol + 1 * 32 + cc, l1);
                tmem_ld16(tb + lane_base + kAccCol + 2 * 32 + cc, l2);
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    v[j] = rs0 * csc[sg * 64 + cc + j] *
                           ((l0[j] + l1[j] * (1.f / 256.f)) + l2[j] * (1.f / 65536.f));
                if (tangent) {
                    tmem_ld16(tb + lane_base + kAccCol + 3 * 32 + cc, l0);
                    tmem_ld16(tb + lane_base + kAccCol + 4 * 32 + cc, l1);
                    tmem_ld16(tb + lane_base + kAccCol + 5 * 32 + cc, l2);
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        v[j] += rs1 * csc[sg * 64 + 32 + cc + j] *
                                ((l0[j] + l1[j] * (1.f / 256.f)) + l2[j] * (1.f / 65536.f));
                }
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const unsigned col = (unsigned)(cc + j);
                staging[((col * 32u + bb) << 2) + p] = v[j];
            }
            if constexpr (BWD) {
                float lo[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float hi = tf32_rna(v[j]);
                    lo[j] = tf32_rna(v[j] - hi);
                    v[j] = hi;
                }
                tmem_st16(tb + lane_base + kAccCol + 0 * 32 + cc, v);
                tmem_st16(tb + lane_base + kAccCol + 1 * 32 + cc, lo);
                tmem_wait_st();
                tc_fence_before();
                mbar_arrive(&bars[B_CREADY]);
            }
            tc_fence_before();
            mbar_arrive(&bars[B_ACCFREE]);
            workers_sync();   // the staging tile is complete

            // Staging -> global (overlaps the environment GEMM and the next tile's MMAs).
            if (!(BWD && (a.mode & TCB_NO_STORE))) {
                const unsigned sw = ub;
                const long long c0 = tile * TN;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const long long c = c0 + 4 * uq + k;
                    if (c < ncols) {
                        const unsigned col = (unsigned)(4 * uq + k);
                        const float4 o = *reinterpret_cast<const float4*>(staging + ((col * 32u + sw) << 2));
                        __stcs(&a.xout[amp_index(c, ub, n, bl)], o);
                    }
                }
            }
            if constexpr (BWD) {
                wait(B_DONE_E, (unsigned)(i & 1));
                workers_sync();
                if (ctl[1]) { ok = false; break; }
                tc_fence_after();
                float e[32];
                tmem_ld32(tb + lane_base + kEnvCol + 64 * (warp >> 2), e);
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[j] += e[j];
                tmem_ld32(tb + lane_base + kEnvCol + 64 * (warp >> 2) + 32, e);
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[32 + j] += e[j];
                tc_fence_before();
                if (++since_flush == kFlushTiles) flush();
            }
            workers_sync();   // the staging tile is reused by the next iteration
        }
        if (ok && BWD && (since_flush > 0 || !flushed)) flush();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (mma_warp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tb), "r"(kTmemCols));
}

}  // namespace

int tcb_tiles(long long ncols, bool /*bwd*/) { return (int)((ncols + TN - 1) / TN); }

cudaError_t tcb_set_smem_limits() {
    cudaError_t e = cudaFuncSetAttribute(tcb_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)launch_smem(false));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(tcb_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)launch_smem(true));
}

cudaError_t launch_tcb(const TcbArgs& a, bool bwd, int ctas, cudaStream_t st) {
    if (a.n < 5 || a.a < 0 || a.a + 5 > a.n || ctas < 1) return cudaErrorInvalidValue;
    const unsigned smem = launch_smem(bwd);
    if (bwd) tcb_kernel<true><<<ctas, kT + 32, smem, st>>>(a);
    else tcb_kernel<false><<<ctas, kT + 32, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace hvp
