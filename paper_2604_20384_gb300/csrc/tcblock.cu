// Tensor-core passes of the fused-block schedule (sm_103a: tcgen05, TMEM).
//
// A pass applies one block of five neighbouring qubits (up to ~10 gates fused
// into a dense 32 x 32 complex operator B and its tangent dB, App. D's
// [[B, 0], [dB, B]]) to every amplitude of every sample. Amplitudes are
// grouped into tiles of 32 block amplitudes x 32 "columns" (the other n - 5
// qubits and the sample). Per tile, the pass is one real GEMM
//     D = [B ; dB] [psi | dpsi]          (128 x 64 times 64 x 64)
// on the real embedding (K = 2 b + re / im of the block index b): the
// operator's rows are those of B over those of dB, the GEMM's columns the
// tile's states over its tangents, so that D holds B psi and B dpsi over
// dB psi (and dB dpsi, unused); psi' = B psi and dpsi' = B dpsi + dB psi.
// Backward the same with B^dag, dB^dag on the co-states (c, dc) (Eq. bis,
// Eq. dbis).
//
// Exact-integer split. The tensor cores' FP32 accumulation truncates, and a
// truncation per accumulation step biases every block application towards
// smaller magnitudes; over the tens of blocks of a sweep that bias exceeds the
// error budget. So each operand is split into three slices of 8-bit integers
// on a power-of-two scale (per row of the operator, per GEMM column of X),
// x = scale * (s_0 + s_1 / 256 + s_2 / 65536) to 2^-25 of the scale; the
// products of slices and their sums over K = 64 are integers below 2^24,
// which the bf16 MMAs (kind::f16, FP32 accumulation) produce exactly. Levels
// i + j = 0, 1, 2 of slice products go to three TMEM accumulators, combined in
// the epilogue with round-to-nearest FP32 arithmetic:
//     D = rs * cs * ((L_0 + L_1 / 256) + L_2 / 65536).
// The operator's three slices sit in TMEM for the whole launch (the A operand
// of tcgen05.mma may come from TMEM); the slices of X are staged in shared
// memory as K-major operands, two slots deep.
//
// Backward, the block environment P = D Psi^T (the co-states at the block's
// input, rows 4 b + p for p = re c, im c, re dc, im dc, against the forward
// states at the block's input, contracted over the tile's columns) is a
// second GEMM on TF32 high and low parts of both operands in shared memory
// (three products), issued after the tile's co-states are complete. The
// results of two consecutive tiles accumulate in TMEM, then are added to
// per-thread FP32 sums (round to nearest) and flushed into the CTA's FP64
// record every 64 such pairs, so the truncating accumulation spans two
// tiles (24 MMAs).
//
// Pipeline. One CTA per SM, 17 warps: warps 0-7 (producers) slice the X
// tiles and, backward, read the environment; warps 8-15 (epilogue) combine
// the accumulators, store the tile and, backward, write the environment
// GEMM's TF32 operands; warp 16 owns TMEM, and its first lane issues every
// MMA and every TMA load of the input ring (four 16 KB slots: forward four X
// tiles, backward two X and two forward-state tiles), refilling a slot once
// the barrier its readers arrive on (FULL, CREADY) shows that they are done
// with it. A tile's slices are staged one iteration before its MMAs.
// Forward, two accumulator buffers let the MMAs of tile i + 1 run during the
// epilogue of tile i;
// backward (one accumulator buffer beside the environment), the environment
// MMAs of tile i - 1 are issued after the update MMAs of tile i and fill the
// tensor pipe while the epilogue of tile i runs. Every wait on an mbarrier is
// bounded: a wait that gives up sets bit 2 of *status, the CTA leaves its
// loop together, commits its MMAs in flight to a separate barrier and waits
// (bounded) for it, then frees its TMEM.
#include "internal.h"

namespace hvp {

namespace {

constexpr int kT = 512;                      // worker threads: producers (warps 0-7), epilogue (warps 8-15)
constexpr int TN = 32;                       // columns per tile
constexpr int NE = 2 * TN;                   // GEMM columns per tile: the states, then the tangents
constexpr unsigned kTmemCols = 512;
constexpr unsigned kOpCol = 0;               // operator slices: 3 x 32 columns (K = 64 bf16 per lane)
constexpr unsigned kAccCol = 96;             // accumulator buffer b at kAccCol + b kAccBuf: levels 0..2
constexpr unsigned kAccBuf = 3 * NE;         //   of NE columns each
constexpr unsigned kEnvCol = kAccCol + kAccBuf;  // backward (one buffer): environment, 128 columns
constexpr unsigned kSumCol = kEnvCol + 128;      // backward: FP32 running sums of environment columns
                                                 //   16..63 of each producer thread's 64 (96 columns)
constexpr int kFlushTiles = 64;              // environment reads summed in FP32 before an FP64 flush
constexpr unsigned kWaitLimit = 1u << 22;    // mbarrier polls before a wait gives up
constexpr unsigned kSettleLimit = 1u << 16;  // polls for an outstanding copy on the way out

// X slices: K = 64 x NE columns, bf16, K-major core matrices (8 columns x 16
// bytes). K-cores 144 bytes apart (a 16-byte gap, so that a warp's 4-byte
// stores of 32 block indices of one column hit 32 banks), column cores 1152.
constexpr unsigned kLboX = 144, kSboX = 1152;
constexpr unsigned kXRegion = (NE / 8) * kSboX;   // one slice
constexpr unsigned kXSlot = 3 * kXRegion;
// Backward, the TF32 operands of the environment GEMM (rows 4 b + p x K = the
// tile's 32 columns): K-cores (4 columns) 128 bytes apart, row cores 1040
// (65 16-byte units, so that eight lanes' 16-byte stores land in eight bank
// groups).
constexpr unsigned kLboE = 128, kSboE = 1040;
constexpr unsigned kERegion = 16 * kSboE;         // one TF32 part (high or low)
// The epilogue's output tile: float4 of (block index b, column c) at b * 33
// + c (rows of 32 columns padded to 33, so that 32 block indices reading
// one column hit distinct bank groups).
constexpr unsigned kRowF4 = 33;
constexpr unsigned kStagingBytes = 32 * kRowF4 * 16;
constexpr unsigned kStaging2Bytes = 32 * kRowF4 * 8;   // dB psi (dB^dag c): float2 per (block index, column)
// Ring of raw input tiles filled by TMA tile loads: forward 4 tiles of X;
// backward 2 of X (co-states) and 2 of the forward states Psi, so that
// several tiles' loads are in flight per SM. A raw tile is four 4 KB boxes
// of 8 columns each (see tile_off).
constexpr unsigned kRawTile = TN * 32 * 16;
__host__ __device__ constexpr int ring_x(bool bwd) { return bwd ? 2 : 4; }
__host__ __device__ constexpr int ring_p(bool bwd) { return bwd ? 2 : 0; }

// Barriers in shared memory (mbarriers):
enum : int {
    B_FULL0 = 0,    // X slot 0 staged (256 producer arrivals)
    B_FULL1 = 1,    // X slot 1 staged
    B_XDONE0 = 2,   // the update MMAs that read X slot 0 complete (commit)
    B_XDONE1 = 3,   // ... X slot 1
    B_DONE0 = 4,    // update MMAs into accumulator buffer 0 complete (commit)
    B_DONE1 = 5,    // ... buffer 1
    B_FREE0 = 6,    // the epilogue has read accumulator buffer 0 (256 arrivals)
    B_FREE1 = 7,    // ... buffer 1
    B_CREADY = 8,   // backward: the tile's co-states are in the TF32 buffer (256 epilogue arrivals)
    B_PREADY = 9,   // backward, even tiles: the previous pair's environment is read (256 producer
                    //   arrivals), so that the tile's environment may start afresh
    B_DONE_E = 10,  // backward: the environment MMAs of an even tile complete (commit)
    B_DRAIN = 11,   // every MMA issued so far complete (commit, on the way out after a failed wait)
    B_RING0 = 12,   // ring slot s (B_RING0 + s, 4 slots): every producer's copies into it complete
    B_SCALES0 = 16, // column scales of tile j in scale slot j mod 4 (B_SCALES0 + slot; 8 producer warps)
    B_DONE_E1 = 20, // backward: the environment MMAs of an odd tile complete (commit)
    B_COUNT = 21
};

// Shared-memory layout (bytes, from a 1024-byte aligned base): the raw-tile
// ring; X slots [2][3 slices]; backward: the forward-state buffer [high,
// low], the co-state buffer [high, low]; staging; column scales [4 slots]
// [NE]; barriers; TMEM base and stop flag.
__host__ __device__ constexpr unsigned off_x(bool bwd) { return (unsigned)(ring_x(bwd) + ring_p(bwd)) * kRawTile; }
__host__ __device__ constexpr unsigned off_psi(bool bwd) { return off_x(bwd) + 2 * kXSlot; }
__host__ __device__ constexpr unsigned off_dbuf(bool bwd) { return off_psi(bwd) + (bwd ? 2 * kERegion : 0u); }
__host__ __device__ constexpr unsigned off_stg(bool bwd) { return off_dbuf(bwd) + (bwd ? 2 * kERegion : 0u); }
__host__ __device__ constexpr unsigned off_stg2(bool bwd) { return off_stg(bwd) + kStagingBytes; }
__host__ __device__ constexpr unsigned off_csc(bool bwd) { return off_stg2(bwd) + kStaging2Bytes; }
__host__ __device__ constexpr unsigned off_bars(bool bwd) { return off_csc(bwd) + 4 * NE * 4; }
__host__ __device__ constexpr unsigned smem_bytes(bool bwd) { return off_bars(bwd) + B_COUNT * 8 + 16 + 1024; }
// Dynamic shared memory of a launch: at least 116 KB, so that one CTA runs
// per SM (it holds all of the SM's TMEM).
constexpr unsigned launch_smem(bool bwd) { return smem_bytes(bwd) > 116u * 1024u ? smem_bytes(bwd) : 116u * 1024u; }
static_assert(smem_bytes(true) <= 227u * 1024u, "shared memory");
static_assert(kSumCol + 96 <= kTmemCols && kAccCol + 2 * kAccBuf <= kTmemCols, "TMEM");

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// kind::tf32 / kind::f16 with bf16 operands, FP32 accumulator, both operands
// K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_tf32(int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_bf16(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// D (TMEM) (+)= A (TMEM) B (shared memory), bf16 operands.
__device__ __forceinline__ void mma_ts_f16(unsigned d, unsigned a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n"
                 :: "r"(d), "r"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
// D (TMEM) (+)= A (shared memory) B (shared memory), TF32 operands.
__device__ __forceinline__ void mma_ss_tf32(unsigned d, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

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
// Three x16 loads at columns taddr, taddr + stride, taddr + 2 stride, one wait.
__device__ __forceinline__ void tmem_ld16x3(unsigned taddr, unsigned stride, float (&a)[16], float (&b)[16],
                                            float (&c)[16]) {
    uint32_t r[48];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%48];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31},"
        " [%49];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47},"
        " [%50];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
          "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
          "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47])
        : "r"(taddr), "r"(taddr + stride), "r"(taddr + 2 * stride)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        a[i] = __uint_as_float(r[i]);
        b[i] = __uint_as_float(r[16 + i]);
        c[i] = __uint_as_float(r[32 + i]);
    }
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
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// One bounded poll of an mbarrier phase: the thread may sleep up to about a
// microsecond (woken early when the phase completes).
__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned par) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(par), "r"(1000u)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// TMA tile load of a 3- or 4-dimensional box (coordinates innermost first).
__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* map, int x0, int x1, int x2, int x3,
                                         uint64_t* bar, bool four) {
    if (four)
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
            "%5}], [%6];" ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x0), "r"(x1), "r"(x2),
            "r"(x3), "r"(smem_u32(bar))
            : "memory");
    else
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
            "%4}], [%5];" ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x0), "r"(x1), "r"(x2),
            "r"(smem_u32(bar))
            : "memory");
}
// Barriers of one role's 256 threads (id 1: producers, id 2: epilogue); the
// second returns the OR of every participant's flag, the same in every thread.
__device__ __forceinline__ void group_sync(int id) { asm volatile("bar.sync %0, 256;" ::"r"(id) : "memory"); }
__device__ __forceinline__ bool group_sync_or(int id, bool v) {
    unsigned r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %2, 0;\n\tbar.red.or.pred q, %1, 256, p;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(r)
                 : "r"(id), "r"((unsigned)v)
                 : "memory");
    return r != 0;
}

// Global amplitude index of block index b and column c (c = the sample and
// the other n - 5 qubits in address order): the block's five bits inserted
// into c at bit bl.
__device__ __forceinline__ size_t amp_index(long long c, unsigned b, int bl) {
    const unsigned long long u = (unsigned long long)c;
    return (size_t)(((u >> bl) << (bl + 5)) | ((unsigned long long)b << bl) | (u & ((1ull << bl) - 1ull)));
}


// Power-of-two scale exponent of a column: 2^e > m >= 2^(e-1) for the largest
// magnitude m (bits of a non-negative float); bounded below so that the
// up-scale 2^(8-e) stays a normal float.
__device__ __forceinline__ int col_exp(unsigned mbits) {
    if (mbits == 0u) return -100;
    const int e = (int)((mbits >> 23) & 255u) - 126;
    return e < -100 ? -100 : e;
}
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((unsigned)(k + 127) << 23); }

// Three 8-bit integer slices of re and im (|.| < 256), y = s0 + s1 / 256 +
// s2 / 65536 up to 2^-17, packed as bf16 pairs (re in the low half; exact).
__device__ __forceinline__ void slice3_pair(float re, float im, uint32_t& p0, uint32_t& p1, uint32_t& p2) {
    const float r0 = rintf(re), i0 = rintf(im);
    const float rr = (re - r0) * 256.f, ir = (im - i0) * 256.f;
    const float r1 = rintf(rr), i1 = rintf(ir);
    const float r2 = rintf((rr - r1) * 256.f), i2 = rintf((ir - i1) * 256.f);
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(p0) : "f"(i0), "f"(r0));
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(p1) : "f"(i1), "f"(r1));
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(p2) : "f"(i2), "f"(r2));
}

// Offset of column c of block index b in a raw tile: four 4 KB boxes of 8
// columns (c = 8 g + c'). At bl >= 3 box g row b holds the 8 columns of block
// index b (128 bytes, 16-byte chunk c' XOR (b mod 8), the TMA's 128-byte
// swizzle); at bl < 3 box g holds 8 / 2^bl runs of 32 x 2^bl amplitudes in
// memory order. Either way the 32 block indices of one column are
// conflict-free for bl = 0 and bl >= 3 (2- and 4-way at bl = 1, 2).
__device__ __forceinline__ unsigned raw_off(unsigned b, unsigned c, int bl) {
    const unsigned g = c >> 3, cq = c & 7u;
    if (bl >= 3) return g * 4096u + b * 128u + ((cq ^ (b & 7u)) << 4);
    const unsigned pl = 1u << bl;
    return g * 4096u + (((cq >> bl) * 32u + b) * pl + (cq & (pl - 1u))) * 16u;
}

// Raw tile loaded by the threads of a role (inputs without a tensor map):
// the thread's four elements (block index b, columns 4 qd .. 4 qd + 3, zero
// past the last column) stored at their raw-tile offsets, then its arrival on
// the slot's barrier. Out of line: the tensor-map path is the usual one.
__device__ __noinline__ void load_raw_direct(unsigned char* dst, const float4* __restrict__ src, long long c0,
                                             long long ncols, unsigned qd, unsigned b, int bl, uint64_t* bar) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const unsigned c = 4u * qd + (unsigned)i;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c0 + c < ncols) v = __ldcs(src + amp_index(c0 + c, b, bl));
        *reinterpret_cast<float4*>(dst + raw_off(b, c, bl)) = v;
    }
    mbar_arrive(bar);   // (release: orders the stores above)
}

// The four TMA box loads of one raw tile (kRawTile bytes expected on bar).
__device__ __forceinline__ void tma_tile(unsigned char* dst, const CUtensorMap* map, long long c0, int bl,
                                         uint64_t* bar) {
    mbar_arrive_expect_tx(bar, kRawTile);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long long cg = c0 + 8 * q;
        if (bl >= 3)
            tma_load(dst + 4096 * q, map, 0, (int)((cg & ((1ll << bl) - 1)) >> 3), 0, (int)(cg >> bl), bar, true);
        else
            tma_load(dst + 4096 * q, map, 0, 0, (int)(cg >> bl), 0, bar, false);
    }
}
// One producer's part of the X operand of a tile: for each of its four
// columns c = 4 uq + i (and, with tangents, TN + c) the power-of-two scale
// from the warp's maximum magnitude (published in cs by lane 0), then the
// three 8-bit slice pairs of its block-index row, stored in the three slice
// regions of xb at kb + the column's core-matrix offset.
__device__ __forceinline__ void slice_cols_body(unsigned char* xb, float* cs, unsigned kb, int uq, int lane,
                                                bool tangent, const float4 (&xr)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int c = 4 * uq + i;
        const unsigned m0 = __reduce_max_sync(0xffffffffu, __float_as_uint(fmaxf(fabsf(xr[i].x), fabsf(xr[i].y))));
        const int e0 = col_exp(m0);
        const float u0 = pow2f(8 - e0);
        uint32_t p0, p1, p2;
        const unsigned o0 = kb + (unsigned)(c & 7) * 16u + (unsigned)(c >> 3) * kSboX;
        slice3_pair(xr[i].x * u0, xr[i].y * u0, p0, p1, p2);
        *reinterpret_cast<uint32_t*>(xb + o0) = p0;
        *reinterpret_cast<uint32_t*>(xb + kXRegion + o0) = p1;
        *reinterpret_cast<uint32_t*>(xb + 2 * kXRegion + o0) = p2;
        if (lane == 0) cs[c] = pow2f(e0 - 8);
        if (tangent) {
            const int cn = TN + c;
            const unsigned m1 = __reduce_max_sync(0xffffffffu, __float_as_uint(fmaxf(fabsf(xr[i].z), fabsf(xr[i].w))));
            const int e1 = col_exp(m1);
            const float u1 = pow2f(8 - e1);
            const unsigned o1 = kb + (unsigned)(cn & 7) * 16u + (unsigned)(cn >> 3) * kSboX;
            slice3_pair(xr[i].z * u1, xr[i].w * u1, p0, p1, p2);
            *reinterpret_cast<uint32_t*>(xb + o1) = p0;
            *reinterpret_cast<uint32_t*>(xb + kXRegion + o1) = p1;
            *reinterpret_cast<uint32_t*>(xb + 2 * kXRegion + o1) = p2;
            if (lane == 0) cs[cn] = pow2f(e1 - 8);
        }
    }
}
// The same out of line, with its inputs by value. The backward kernel's
// four roles do not fit the instruction cache together, and it runs faster
// with its producers' slicing as a call (the forward kernel, with less code,
// runs faster with it inlined).
template <bool TAN>
__device__ __noinline__ void slice_cols_call(unsigned char* xb, float* cs, unsigned kb, int uq, int lane,
                                             float4 x0, float4 x1, float4 x2, float4 x3) {
    const float4 xr[4] = {x0, x1, x2, x3};
    slice_cols_body(xb, cs, kb, uq, lane, TAN, xr);
}

// The retry loop of a bounded wait, out of line (the first try stays inline):
// polls until the phase completes, the stop flag rises or the limit runs
// out, which raises the stop flag and sets bit 2 of *status.
__device__ __noinline__ bool wait_retry(uint64_t* bar, unsigned par, volatile unsigned* ctl, unsigned limit,
                                        int* status) {
    for (unsigned i = 0; i < limit; ++i) {
        if (mbar_try(bar, par)) return true;
        if ((i & 255u) == 255u && ctl[1]) return false;
    }
    ctl[1] = 1u;
    atomicOr(status, 2);
    return false;
}

// Rows 4 b + p (p = the four components, four columns per 16-byte row) of a
// TF32 operand of the environment GEMM: high parts at dst + base, low parts
// one region further. One copy of this code serves both operands.
__device__ __noinline__ void put_tf32_rows(unsigned char* dst, unsigned base, float4 v0, float4 v1, float4 v2,
                                           float4 v3) {
    const float4 v[4] = {v0, v1, v2, v3};
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        float h[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float x = p == 0 ? v[i].x : p == 1 ? v[i].y : p == 2 ? v[i].z : v[i].w;
            h[i] = tf32_rna(x);
            l[i] = tf32_rna(x - h[i]);
        }
        *reinterpret_cast<float4*>(dst + base + 16 * p) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4*>(dst + kERegion + base + 16 * p) = make_float4(l[0], l[1], l[2], l[3]);
    }
}

template <bool BWD, bool TAN>
__global__ void __launch_bounds__(kT + 32) tcb_kernel(const __grid_constant__ TcbArgs a) {
    constexpr int NB = BWD ? 1 : 2;   // accumulator buffers
    constexpr int RX = ring_x(BWD), RP = ring_p(BWD);
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* base = smem + ((1024u - (smem_u32(smem) & 1023u)) & 1023u);   // 1024-byte aligned
    unsigned char* ring = base;
    unsigned char* xslots = base + off_x(BWD);
    unsigned char* psislots = base + off_psi(BWD);
    unsigned char* dbuf = base + off_dbuf(BWD);
    float* staging = reinterpret_cast<float*>(base + off_stg(BWD));
    float* staging2 = reinterpret_cast<float*>(base + off_stg2(BWD));
    float* csc = reinterpret_cast<float*>(base + off_csc(BWD));
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + off_bars(BWD));
    volatile unsigned* ctl = reinterpret_cast<volatile unsigned*>(bars + B_COUNT);   // [TMEM base, stop]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool mma_warp = warp == 16, producer = warp < 8;
    const int n = a.n, bl = n - a.a - 5;
    const long long ncols = a.ncols;
    const long long ntiles = (ncols + TN - 1) / TN;
    const long long g = gridDim.x;
    const unsigned limit = a.wait_limit ? a.wait_limit : kWaitLimit;
    // the tangent components are carried (else zero and left out): fixed at
    // compile time in the backward kernel, read from the mode forward
    const bool tangent = BWD ? TAN : !(a.mode & TCB_NO_TANGENT);
    const int dir = BWD ? 1 : 0;

    if (mma_warp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void*)ctl)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        const unsigned cm = 1u + a.barrier_extra;   // arrivals a commit barrier expects
        // ring slots: one arrival (the TMA issuer, expecting the bytes) or,
        // for inputs loaded by the threads (no tensor map), one per thread of the role
        const bool xgen = !a.tma_x, pgen = !a.tma_p;
        const unsigned rx = xgen ? 256u : 1u, rp = pgen ? 256u : 1u;
        const unsigned r2 = RX > 2 ? rx : rp, r3 = RX > 3 ? rx : rp;
        const unsigned counts[B_COUNT] = {256u, 256u, cm, cm, cm, cm, 256u, 256u, 256u, 256u,
                                          cm, 1u, rx, rx, r2, r3, 8u, 8u, 8u, 8u, cm};
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
    const int row = (warp & 3) * 32 + lane;   // TMEM lane of this thread (worker warps)

    // Operator slices into TMEM: warps 0-3 slices 0 and 1, warps 4-7 slice 2;
    // each thread its row (32 words = 64 bf16 per slice).
    if (producer) {
        for (int i = (warp < 4 ? 0 : 2); i < (warp < 4 ? 2 : 3); ++i) {
            const uint32_t* src = a.ops + (dir * 3 + i) * kOpSliceWords + row * 32;
            uint32_t v[32];
#pragma unroll
            for (int w = 0; w < 32; ++w) v[w] = __ldg(&src[w]);
            tmem_st32u(tb + lane_base + kOpCol + i * 32, v);
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
        if constexpr (BWD) {   // (less code: the backward kernel overflows the instruction cache)
            if (mbar_try(&bars[b], par)) return true;
            return wait_retry(&bars[b], par, ctl, limit, a.status);
        } else {
            for (unsigned i = 0; i < limit; ++i) {
                if (mbar_try(&bars[b], par)) return true;
                if ((i & 255u) == 255u && ctl[1]) return false;
            }
            ctl[1] = 1u;
            atomicOr(a.status, 2);
            return false;
        }
    };

    // ------------------------------------------------------------ input ring
    // Read by the producers (X) and, backward, by the epilogue (Psi): a
    // worker thread's elements are block index lane, columns 4 qd .. 4 qd + 3
    // (qd its warp's column quad).
    const int qd = warp < 8 ? warp : warp - 8;
    bool bad = false;
    auto tile_off = [&](unsigned b, unsigned c) -> unsigned { return raw_off(b, c, bl); };
    // Loads of local tile j (global tile blockIdx.x + j gridDim.x) into its
    // ring slot (X: j mod RX; Psi: RX + j mod RP). With a tensor map the MMA
    // warp's issuing lane loads the ring (issue_tma): the first tiles at the
    // start, then each X slot again once every producer has staged the tile
    // it held (FULL), each Psi slot once every epilogue thread has staged
    // its forward states (CREADY), so that no worker thread issues copies.
    // Without one, the role's threads load their own elements when the slot
    // is free (after the role's barrier), each arriving on the slot's
    // barrier. Nothing is issued for tiles past the end (no one waits for
    // them).
    long long x_issued = 0, p_issued = 0;   // local tiles issued by the MMA lane
    auto issue_tma = [&](long long j, bool psi) {
        const long long tile = (long long)blockIdx.x + j * g;
        if (tile >= ntiles) return;
        const int s = psi ? RX + (int)(j % (RP > 0 ? RP : 1)) : (int)(j % RX);
        (psi ? p_issued : x_issued) = j + 1;
        unsigned char* dst = ring + (unsigned)s * kRawTile;
        const CUtensorMap* map = psi ? &a.tm_p : &a.tm_x;
        tma_tile(dst, map, tile * TN, bl, &bars[B_RING0 + s]);
    };
    auto issue_direct = [&](long long j, int s, bool psi) {
        const long long tile = (long long)blockIdx.x + j * g;
        if (tile >= ntiles) return;
        load_raw_direct(ring + (unsigned)s * kRawTile, psi ? a.psi : a.xin, tile * TN, ncols, (unsigned)qd,
                        (unsigned)lane, bl, &bars[B_RING0 + s]);
    };
    auto issue_x = [&](long long j) {
        if (!a.tma_x) issue_direct(j, (int)(j % RX), false);
    };
    auto issue_p = [&](long long j) {
        if (!a.tma_p) issue_direct(j, RX + (int)(j % (RP > 0 ? RP : 1)), true);
    };
    // The thread's four raw values of local tile j (zero past the last
    // column), once the slot is full.
    auto take = [&](long long j, int s, int uses, float4 (&v)[4]) {
        if (!wait(B_RING0 + s, (unsigned)(uses & 1))) bad = true;
        const unsigned char* src = ring + (unsigned)s * kRawTile;
        const long long c0 = ((long long)blockIdx.x + j * g) * TN;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const unsigned c = (unsigned)(4 * qd + i);
            v[i] = *reinterpret_cast<const float4*>(src + tile_off((unsigned)lane, c));
            if (c0 + c >= ncols) v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (!tangent) { v[i].z = 0.f; v[i].w = 0.f; }
        }
    };
    // No copy into shared memory outlives the CTA: the MMA lane waits for its
    // last copy into each ring slot (bounded, regardless of the stop flag);
    // every earlier copy into the slot was taken before the next was issued.
    auto settle = [&](long long from, long long to, int base, int depth) {
        for (long long q = from; q < to; ++q)
            for (unsigned k = 0; k < kSettleLimit; ++k)
                if (mbar_try(&bars[B_RING0 + base + (int)(q % depth)], (unsigned)((q / depth) & 1))) break;
    };

    if (mma_warp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t id_u = idesc_bf16(tangent ? NE : TN), id_e = idesc_tf32(128);
            const unsigned xs0 = smem_u32(xslots);
            const uint64_t kx = (uint64_t)((2u * kLboX) >> 4), ke = (uint64_t)((2u * kLboE) >> 4);
            // P = D Psi^T of one tile: K = its 32 columns, 4 K-steps of 8;
            // high x high + high x low + low x high. The environments of two
            // consecutive tiles (local 2m and 2m + 1) accumulate in TMEM
            // before the producers read them.
            auto env = [&](bool onto, int done) {
                const unsigned ps = smem_u32(psislots), ds = smem_u32(dbuf);
                const uint64_t ph = sdesc(ps, kLboE, kSboE), pl = sdesc(ps + kERegion, kLboE, kSboE);
                const uint64_t dh = sdesc(ds, kLboE, kSboE), dl = sdesc(ds + kERegion, kLboE, kSboE);
#pragma unroll
                for (int k = 0; k < TN / 8; ++k) {
                    mma_ss_tf32(tb + kEnvCol, dh + k * ke, ph + k * ke, id_e, onto || k > 0);
                    mma_ss_tf32(tb + kEnvCol, dh + k * ke, pl + k * ke, id_e, 1);
                    mma_ss_tf32(tb + kEnvCol, dl + k * ke, ph + k * ke, id_e, 1);
                }
                mma_commit(&bars[done]);
            };
            // the environment of tile j once its co-states and forward states are staged
            auto env_of = [&](long long j) -> bool {
                if (!wait(B_CREADY, (unsigned)(j & 1))) return false;
                if (a.tma_p) issue_tma(j + RP, true);   // every epilogue thread has read Psi slot j mod RP
                if ((j & 1) == 0 && !wait(B_PREADY, (unsigned)((j >> 1) & 1))) return false;
                tc_fence_after();
                env((j & 1) != 0, (j & 1) ? B_DONE_E1 : B_DONE_E);   // odd tiles add onto the even tile before them
                return true;
            };
            if (a.tma_x)   // the ring's first tiles
                for (int q = 0; q < RX; ++q) issue_tma(q, false);
            if (BWD && a.tma_p)
                for (int q = 0; q < RP; ++q) issue_tma(q, true);
            bool issued = false, ok = true;
            long long i = 0;
            for (long long tile = blockIdx.x; tile < ntiles; tile += g, ++i) {
                const int sg = (int)(i & 1), ab = NB == 2 ? sg : 0;
                if (!wait(B_FULL0 + sg, (unsigned)((i >> 1) & 1))) { ok = false; break; }
                if (a.tma_x) issue_tma(i + RX, false);   // every producer has read X slot i mod RX
                if (i >= NB && !wait(B_FREE0 + ab, (unsigned)((i / NB - 1) & 1))) { ok = false; break; }
                tc_fence_after();
                // D = A X: levels 0..2 of slice products (i + j = level), 4 K-steps of 16.
                const unsigned xs = xs0 + sg * kXSlot, acc = tb + kAccCol + ab * kAccBuf;
#pragma unroll
                for (int lev = 0; lev < 3; ++lev) {
#pragma unroll
                    for (int ii = 0; ii <= lev; ++ii) {
                        const uint64_t bd = sdesc(xs + (lev - ii) * kXRegion, kLboX, kSboX);
                        const unsigned ad = tb + kOpCol + ii * 32;
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            mma_ts_f16(acc + lev * NE, ad + 8 * k, bd + k * kx, id_u, (ii | k) != 0);
                    }
                }
                mma_commit(&bars[B_XDONE0 + sg]);
                mma_commit(&bars[B_DONE0 + ab]);
                issued = true;
                if (BWD && i > 0 && !env_of(i - 1)) { ok = false; break; }
            }
            if (BWD && ok && i > 0) env_of(i - 1);
            if (ctl[1] && issued) {   // let every MMA issued so far finish (bounded) before TMEM is freed
                mma_commit(&bars[B_DRAIN]);
                for (unsigned k = 0; k < kWaitLimit; ++k)
                    if (mbar_try(&bars[B_DRAIN], 0u)) break;
            }
            if (a.tma_x) settle(x_issued > RX ? x_issued - RX : 0, x_issued, 0, RX);
            if (BWD && a.tma_p) settle(p_issued > RP ? p_issued - RP : 0, p_issued, RX, RP > 0 ? RP : 1);
        }
        __syncwarp();
    } else if (producer) {
        // ------------------------------------------------------------ producers
        // Warp w owns the tile's column quad w (columns 4w .. 4w + 3), lane l
        // the block index b = l: column maxima are warp reductions.
        const unsigned ub = (unsigned)lane;
        const int uq = warp;
        bool ok = true;
        // Local tile j -> X slot sg: per column (state and tangent part) the
        // scale exponent from the warp maximum (published in scale slot j mod
        // 4), then the slices. (The ring slot is refilled once every producer
        // has read it.)
        auto produce_x = [&](long long j, int sg) {
            float4 xr[4];
            take(j, (int)(j % RX), (int)(j / RX), xr);
            unsigned char* xb = xslots + sg * kXSlot;
            float* cs = csc + (int)(j & 3) * NE;
            const unsigned kb = (ub >> 2) * kLboX + (ub & 3u) * 4u;
            if constexpr (BWD) slice_cols_call<TAN>(xb, cs, kb, uq, lane, xr[0], xr[1], xr[2], xr[3]);
            else slice_cols_body(xb, cs, kb, uq, lane, tangent, xr);
            if (lane == 0) mbar_arrive(&bars[B_SCALES0 + (int)(j & 3)]);
            fence_async_smem();
            mbar_arrive(&bars[B_FULL0 + sg]);
        };
        // Backward: FP32 running sums of the environment, this thread's TMEM
        // lane (row 4 b + p of D) and columns 64 k .. 64 k + 63 (k = w / 4,
        // rows of Psi): the first 16 in registers, the other 48 in TMEM.
        float acc[BWD ? 16 : 1];
#pragma unroll
        for (int i = 0; i < (BWD ? 16 : 1); ++i) acc[i] = 0.f;
        const unsigned envc = tb + lane_base + kEnvCol + 64 * (warp >> 2);
        const unsigned sumc = tb + lane_base + kSumCol + 48 * (warp >> 2);
        auto zero_sums = [&]() {
            if constexpr (BWD) {
                float z[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) z[j] = 0.f;
#pragma unroll
                for (int h = 0; h < 3; ++h) tmem_st16(sumc + 16 * h, z);
                tmem_wait_st();
            }
        };
        zero_sums();
        int since_flush = 0;
        bool flushed = false;
        auto flush = [&]() {
            if constexpr (BWD) {
                double* dst = a.rec + (size_t)blockIdx.x * 16384 + (size_t)row * 128 + 64 * (warp >> 2);
                auto add8 = [&](int off, const float (&t)[16]) {
#pragma unroll
                    for (int i = 0; i < 16; i += 2) {
                        double2* q = reinterpret_cast<double2*>(dst + off + i);
                        double2 o = flushed ? *q : make_double2(0.0, 0.0);
                        o.x += (double)t[i];
                        o.y += (double)t[i + 1];
                        *q = o;
                    }
                };
                add8(0, acc);
#pragma unroll
                for (int h = 0; h < 3; ++h) {
                    float t[16];
                    tmem_ld16(sumc + 16 * h, t);
                    add8(16 + 16 * h, t);
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[i] = 0.f;
                zero_sums();
                flushed = true;
                since_flush = 0;
            }
        };
        auto read_env = [&](bool final) {
            if constexpr (BWD) {
                float e[16], t[16];
                tmem_ld16(envc, e);
#pragma unroll
                for (int k = 0; k < 16; ++k) acc[k] += e[k];
#pragma unroll
                for (int h = 0; h < 3; ++h) {
                    tmem_ld16(envc + 16 + 16 * h, e);
                    tmem_ld16(sumc + 16 * h, t);
#pragma unroll
                    for (int k = 0; k < 16; ++k) t[k] += e[k];
                    tmem_st16(sumc + 16 * h, t);
                }
                tmem_wait_st();
                if (++since_flush == kFlushTiles || final) flush();
            }
        };

        // Producers run one tile ahead: in iteration j they stage X of tile
        // j + 1 (its slot is free once the update MMAs of tile j - 1 are
        // done), then (backward, j - 1 odd) read the environment summed over
        // tiles j - 2 and j - 1, which the tensor pipe ran after the update
        // of tile j, so that the environment of tile j may start afresh.
        // (The last environment is read in one more iteration, j == count,
        // so that the read and its flush exist once in the code.)
        const long long count = (long long)blockIdx.x < ntiles ? (ntiles - blockIdx.x + g - 1) / g : 0;
        if (count > 0) {
            for (int q = 0; q < RX; ++q) issue_x(q);
            produce_x(0, 0);
        }
        if (group_sync_or(1, bad)) ok = false;
        else issue_x(RX);
        for (long long j = 0; ok && j <= count; ++j) {
            const bool last = j == count;
            if (last && !(BWD && count > 0)) break;
            const bool more = j + 1 < count;
            if (more) {
                const int sg = (int)((j + 1) & 1);
                if (j >= 1 && !wait(B_XDONE0 + sg, (unsigned)(((j - 1) >> 1) & 1))) bad = true;
                produce_x(j + 1, sg);
            }
            if (BWD) {
                // the sums are read after each pair of tiles (j - 2, j - 1)
                // and after the last tile, once its environment MMAs are
                // complete (even and odd tiles commit to barriers of their
                // own, so that each is waited for phase by phase); then an
                // even tile's environment may start afresh (PREADY, which
                // never runs two phases ahead of the MMA warp's wait: the
                // next arrival follows the read of an environment issued
                // after that wait)
                if (j >= 1 && (((j - 1) & 1) || last)) {
                    const long long t = j - 1;
                    if (!wait((t & 1) ? B_DONE_E1 : B_DONE_E, (unsigned)((t >> 1) & 1))) bad = true;
                    tc_fence_after();
                    read_env(last);
                }
                if (!last && (j & 1) == 0) {
                    tc_fence_before();
                    mbar_arrive(&bars[B_PREADY]);
                }
            }
            // all leave together if any wait gave up; else every producer has
            // read the ring slots taken above: refill them
            if (group_sync_or(1, bad)) { ok = false; break; }
            if (more) issue_x(j + 1 + RX);
        }
        if (BWD && ok && count == 0) {   // no tiles: this CTA's record is zero
            double* dst = a.rec + (size_t)blockIdx.x * 16384 + (size_t)row * 128 + 64 * (warp >> 2);
            for (int i = 0; i < 64; ++i) dst[i] = 0.0;
        }
    } else {
        // ------------------------------------------------------------ epilogue
        // Thread = TMEM lane = operator row. Rows 0-63 (warps with w % 4 < 2)
        // are B's: the state part of the GEMM columns gives psi' (c'), the
        // tangent part B dpsi (B^dag dc); rows 64-127 are dB's, of which the
        // state part (dB psi, dB^dag c) is read. Chunks of 16 accumulator
        // columns per warp: B rows 32 (state part for e = w - 8 < 4, tangent
        // part for e >= 4), dB rows 16.
        const int e = warp - 8;
        const float rs = __ldg(reinterpret_cast<const float*>(a.ops + kOpScaleOff) + dir * 128 + row);
        const bool brow = (warp & 3) < 2;
        const int nchunk = tangent ? (brow ? 2 : 1) : (brow ? 1 : 0);
        const int cb0 = tangent ? (brow ? 32 * (e >> 2) : 16 * (e >> 2)) : 16 * (e >> 2);
        const unsigned bq = (unsigned)(row & 63) >> 1, qc = (unsigned)row & 1u;
        const int bm = bl < 5 ? bl : 5;
        auto combine = [&](unsigned accb, int cb, const float* cs, float (&v)[16]) {
            float t[16], u[16];
            tmem_ld16x3(accb + lane_base + cb, NE, v, t, u);
            const float4* cs4 = reinterpret_cast<const float4*>(cs + cb);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 c4 = cs4[q];
                const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int k = 4 * q + r;
                    v[k] = rs * cv[r] * ((v[k] + t[k] * (1.f / 256.f)) + u[k] * (1.f / 65536.f));
                }
            }
        };
        // Staging: float4 of (block index b, column c) at b * 33 + c (B rows:
        // psi' and B dpsi), float2 at b * 33 + c (dB rows: dB psi), added
        // when the tile is read.
        auto put = [&](int cb, const float (&v)[16]) {
            const unsigned p = (cb >= TN ? 2u : 0u) + qc;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const unsigned c = (unsigned)(cb + k) & (TN - 1);
                staging[((bq * kRowF4 + c) << 2) + p] = v[k];
                if (!tangent) staging[((bq * kRowF4 + c) << 2) + 2 + qc] = 0.f;
            }
        };
        auto put_dB = [&](int cb, const float (&v)[16]) {
#pragma unroll
            for (int k = 0; k < 16; ++k) staging2[((bq * kRowF4 + (unsigned)(cb + k)) << 1) + qc] = v[k];
        };
        const float4* st4 = reinterpret_cast<const float4*>(staging);
        const float2* st2 = reinterpret_cast<const float2*>(staging2);
        auto out = [&](unsigned b, unsigned c) {
            float4 o = st4[b * kRowF4 + c];
            if (tangent) {
                const float2 d = st2[b * kRowF4 + c];
                o.z += d.x;
                o.w += d.y;
            }
            return o;
        };

        // Backward: the forward states of local tile j as the TF32 operand of
        // the environment GEMM (rows 4 b + p, 4 columns per 16-byte row; high
        // and low parts).
        auto produce_psi = [&](long long j) {
            if constexpr (BWD) {
                float4 v[4];
                take(j, RX + (int)(j % RP), (int)(j / RP), v);
                put_tf32_rows(psislots, (unsigned)qd * kLboE + ((unsigned)lane >> 1) * kSboE + ((unsigned)lane & 1u) * 64u,
                              v[0], v[1], v[2], v[3]);
                fence_async_smem();
            }
        };

        if (BWD && (long long)blockIdx.x < ntiles)
            for (int q = 0; q < RP; ++q) issue_p(q);
        long long j = 0;
        for (long long tile = blockIdx.x; tile < ntiles; tile += g, ++j) {
            const int ab = NB == 2 ? (int)(j & 1) : 0;
            if (!wait(B_SCALES0 + (int)(j & 3), (unsigned)((j >> 2) & 1))) bad = true;
            if (!wait(B_DONE0 + ab, (unsigned)((j / NB) & 1))) bad = true;
            tc_fence_after();
            float v[16];
            {
                const unsigned accb = tb + kAccCol + ab * kAccBuf;
                const float* cs = csc + (int)(j & 3) * NE;
                if (nchunk > 1) {
                    combine(accb, cb0, cs, v);
                    put(cb0, v);
                }
                if (nchunk > 0) combine(accb, cb0 + (nchunk - 1) * 16, cs, v);
                tc_fence_before();
                mbar_arrive(&bars[B_FREE0 + ab]);
                if (nchunk > 0) {
                    if (brow) put(cb0 + (nchunk - 1) * 16, v);
                    else put_dB(cb0, v);
                }
            }
            if (group_sync_or(2, bad)) break;
            // staging -> global in memory order (consecutive lanes, 512
            // contiguous bytes per warp instruction for bl >= 5)
            const long long c0 = tile * TN;
            if (!(BWD && (a.mode & TCB_NO_STORE))) {
                if (bm == 5) {   // lane = column, block indices 4 e + k: one base, 2^bl apart
                    if (c0 + lane < ncols) {
                        float4* p = a.xout + amp_index(c0 + lane, 4u * (unsigned)e, bl);
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            __stcs(p + ((size_t)k << bl), out(4u * (unsigned)e + (unsigned)k, (unsigned)lane));
                    }
                } else {
                    const unsigned bmk = (1u << bm) - 1u;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const unsigned f = (unsigned)(32 * (4 * e + k) + lane);
                        const unsigned c = (f & bmk) | ((f >> (bm + 5)) << bm), b = (f >> bm) & 31u;
                        if (c0 + c < ncols) __stcs(&a.xout[amp_index(c0 + c, b, bl)], out(b, c));
                    }
                }
            }
            if constexpr (BWD) {
                // the co-states as the TF32 operand of the environment GEMM,
                // once the previous environment MMAs have read the buffer
                if (j >= 1 && !wait(((j - 1) & 1) ? B_DONE_E1 : B_DONE_E, (unsigned)(((j - 1) >> 1) & 1))) bad = true;
                const unsigned ub = (unsigned)lane;
                const unsigned base = (unsigned)e * kLboE + (ub >> 1) * kSboE + (ub & 1u) * 64u;
                float4 o[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) o[k] = out(ub, (unsigned)(4 * e + k));
                produce_psi(j);
                put_tf32_rows(dbuf, base, o[0], o[1], o[2], o[3]);
                fence_async_smem();
                mbar_arrive(&bars[B_CREADY]);
            }
            group_sync(2);   // the staging tile is reused by the next tile
            if (BWD && !bad) issue_p(j + RP);   // every epilogue thread has read its forward states
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (mma_warp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tb), "r"(kTmemCols));
}

}  // namespace

int tcb_tiles(long long ncols, bool /*bwd*/) { return (int)((ncols + TN - 1) / TN); }

cudaError_t tcb_set_smem_limits() {
    const cudaFuncAttribute attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(tcb_kernel<false, true>, attr, (int)launch_smem(false));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tcb_kernel<true, true>, attr, (int)launch_smem(true));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tcb_kernel<true, false>, attr, (int)launch_smem(true));
    return e;
}

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    }
    return fn;
}

// Tensor map of a state array (float4 per amplitude; column c = the sample
// and the other n - 5 qubits, block bits at bl) whose boxes are the raw
// tiles' 8-column boxes: bl >= 3, dims (8 amplitudes x 4 floats, 2^bl / 8,
// 32 block indices, ncols / 2^bl), box (32, 1, 32, 1), 128-byte swizzle;
// bl < 3, dims (2^bl x 4 floats, 32, ncols / 2^bl), box (4 2^bl, 32, 8 /
// 2^bl), no swizzle. False if the map cannot be made (then the kernel's
// threads load directly).
bool encode_state_map(CUtensorMap* m, const void* base, int bl, long long ncols) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || !base || ncols < 8) return false;
    cuuint64_t dims[4], strides[3];
    cuuint32_t box[4], es[4] = {1, 1, 1, 1};
    cuuint32_t rank;
    CUtensorMapSwizzle sw;
    if (bl >= 3) {
        rank = 4;
        dims[0] = 32; dims[1] = (1ull << bl) / 8; dims[2] = 32; dims[3] = (cuuint64_t)(ncols >> bl);
        strides[0] = 128; strides[1] = 16ull << bl; strides[2] = 16ull << (bl + 5);
        box[0] = 32; box[1] = 1; box[2] = 32; box[3] = 1;
        sw = CU_TENSOR_MAP_SWIZZLE_128B;
    } else {
        rank = 3;
        const unsigned pl = 1u << bl;
        dims[0] = 4 * pl; dims[1] = 32; dims[2] = (cuuint64_t)(ncols >> bl);
        strides[0] = 16ull * pl; strides[1] = 16ull * pl * 32;
        box[0] = 4 * pl; box[1] = 32; box[2] = 8 / pl;
        sw = CU_TENSOR_MAP_SWIZZLE_NONE;
    }
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t launch_tcb(const TcbArgs& args, bool bwd, int ctas, cudaStream_t st) {
    if (args.n < 5 || args.a < 0 || args.a + 5 > args.n || ctas < 1) return cudaErrorInvalidValue;
    TcbArgs a = args;
    const int bl = a.n - a.a - 5;
    a.tma_x = encode_state_map(&a.tm_x, a.xin, bl, a.ncols);
    a.tma_p = bwd && encode_state_map(&a.tm_p, a.psi, bl, a.ncols);
    const unsigned smem = launch_smem(bwd);
    const bool tan = !(a.mode & TCB_NO_TANGENT);
    if (bwd && tan) tcb_kernel<true, true><<<ctas, kT + 32, smem, st>>>(a);
    else if (bwd) tcb_kernel<true, false><<<ctas, kT + 32, smem, st>>>(a);
    else tcb_kernel<false, true><<<ctas, kT + 32, smem, st>>>(a);   // (forward: the mode decides)
    return cudaGetLastError();
}

}  // namespace hvp
