// Hashing on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The projections of a block of 128 points onto all hash rows are the dense
// contraction V = X W^T (K = d_pad <= 320).  The hyperplanes' entries are
// bfloat16 values, so W is exact in bfloat16; the points are split into
// bfloat16 halves X = Xh + Xl (|x - xh - xl| <= 2^-18 |x| per entry) and
//   X W^T ~= Xh W^T + Xl W^T
// (two bfloat16 products, float32 accumulation in tensor memory).  The error
// is below 2^-18 |x||w| for the split plus the float32 accumulation (2 * 4 *
// KB MMAs of 16 exact products, at most 17 float32 roundings of a partial sum
// bounded by |x||w| each, even for a truncating adder): 3.6e-5 |w| for unit x
// and d_pad <= 128, 8.5e-5 |w| up to 320.  The epilogue decides every hash
// bit with the rule of the float64 definition and the row's band, 2^-14 |w| =
// 6.1e-5 |w| (d_pad <= 128) or 2^-12 |w| = 2.4e-4 |w| (params.cpp): a decision
// closer to its boundary than the band is recomputed in float64 in index
// order, which is the defining value (Sec. 2.2: HP bit = [<a,x> >= 0]; CP
// value = sign and index of the largest |<a_c,x>|), so codes are
// bit-identical to the float64 definition.
//
// Kernel structure (one CTA per SM, persistent, warp-specialised; P point
// tiles per work unit: P = 2 for d_pad <= 128, 1 above, where the A tiles of
// two point tiles would not fit in shared memory beside the B ring):
//   - a unit of work is (P point tiles, segment); a segment is one repetition
//     (CP: fns functions of d_pad rows, each cut into N tiles of at most 128
//     rows; HP: a group of 4 repetitions = 128 rows) or a group of 2 sketches
//     (128 rows); while at least G groups of point tiles are left (G = the
//     grid), CTA b takes whole groups b, b + G, ... with all their segments,
//     so the CTAs walk the hash rows in step and each B tile comes from DRAM
//     about once per round and from L2 for the other CTAs; the units of the
//     last groups are split into equal contiguous ranges (the CTAs' shares
//     differ by at most one segment, and each CTA loads the A tiles of only
//     the one or two groups its range touches).  With P = 2 both point tiles
//     are multiplied by every B tile the CTA loads, which halves the B stream;
//   - warp 0 (one thread) is the TMA producer: the A tiles (Xh, Xl of the P
//     point tiles, KB blocks of 64 columns each) once per run of segments,
//     then for every N tile its B operand as KB boxes of 64 columns into a
//     ring of shared-memory stages (as many as fit beside the A tiles, at
//     most 8); all tiles are K-major with the 128-byte swizzle;
//   - warp 1 owns the tensor memory and (one thread) issues the MMAs: per K
//     block and point tile, Xh*W and Xl*W from the stage, into the point
//     tile's 128-column accumulator of one of two buffers (2 buffers x P point
//     tiles x 128 columns, so the epilogue of one N tile overlaps the MMAs of
//     the next); tcgen05.commit frees each stage and publishes each finished
//     accumulator;
//   - four epilogue warps per point tile (one thread per point, tcgen05.ld of
//     its lane quarter = warp % 4) hand each accumulator back through an
//     mbarrier; for a CP function the thread keeps the three largest |v| as
//     integer sort keys in four independent chains (no branches), merged
//     across the function's N tiles; a decision closer to its boundary than
//     the band is queued, with the top two rows as the candidates (or "all
//     rows" when a third row is also close), in the CTA's own region of the
//     request queue (a shared-memory counter, no global atomics);
//   - every mbarrier wait is bounded: on time-out the kernel records an error
//     word and every role leaves its loop.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "pf_internal.h"

namespace pf {

namespace {

constexpr int kBM = 128;          // points per tile (MMA M)
constexpr int kBN = 128;          // rows of an N tile (a CP function of more rows takes several)
// producer warp, MMA warp, 4 epilogue warps per point tile (P point tiles per unit)
constexpr int threads_for(int P) { return 32 * (2 + 4 * P); }
constexpr int kTileBytes = kBM * 128;  // one 64-element K block of 128 rows
constexpr int kMaxStages = 8;     // B ring (fewer when the A tiles leave less shared memory)
constexpr int kSmemLimit = 232448;     // shared memory a CTA may use
// [2 buffers][P point tiles] accumulators of 128 columns
constexpr int tmem_cols_for(int P) { return 2 * P * kBN; }
// point tiles per work unit for a padded dimension
constexpr int pair_for(int d_pad) { return d_pad <= 128 ? 2 : 1; }
constexpr uint32_t kSuspendNs = 5000;        // longest sleep of one try_wait
constexpr uint64_t kWaitNs = 1000000000ull;  // a bounded wait gives up after 1 s
constexpr uint32_t kWaitPolls = 1u << 26;    // ... or after this many polls

struct HashArgs {
  const __nv_bfloat16* xh;
  const __nv_bfloat16* xl;
  const float* x32;
  int64_t npts;
  const __nv_bfloat16* wh;
  const float* w32;
  const float* thr;
  int64_t hash_rows;
  int d, d_pad, KB, family, L, M, fns, ell, rows_table;
  int nsub;        // N tiles per CP function: ceil(d_pad / 128)
  int seg_tables;  // segments that are repetitions (CP) or groups of 4 repetitions (HP)
  int segs;        // + sketch groups of 2
  int64_t units;   // point-tile groups * segs (see Sched for their order)
  int stages;      // B ring stages
  int hold_b;      // diagnostics: issue no B loads, so that the waits on them expire
  uint32_t* codes;
  int64_t cj, cp;
  uint64_t* sk;
  int64_t sm, sp;
  int32_t* error;
  RecheckReq* rq;       // deferred float64 rechecks (may be null): region b = [b*rq_per, (b+1)*rq_per)
  uint32_t* rq_count;   // per region: requests written there (the ones that did not fit ran inline)
  uint32_t rq_per;      // entries per region (0 without a queue)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

// one poll; a thread whose phase is not complete may sleep up to kSuspendNs
// (woken early when the phase completes), so idle roles do not spin on the
// issue slots the epilogue needs
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bounded wait for the phase with the given parity: false once kWaitNs have
// passed (or after kWaitPolls polls, whichever comes first)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < kWaitPolls; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst_smem), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, bf16 inputs, f32 accumulate
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
// 2-D tiled TMA load of box {64 columns, rows} at (x = column, y = row)
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// 16 consecutive 32-bit columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// columns [0, 64) of this thread's lane, waited for
__device__ __forceinline__ void tmem_ld64_x64(uint32_t taddr, uint32_t (&r)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%64];\n"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%65];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
        "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr), "r"(taddr + 32u)
      : "memory");
}

// columns [0, 48); the rest of r reads as zero
__device__ __forceinline__ void tmem_ld64_x48(uint32_t taddr, uint32_t (&r)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%48];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47}, [%49];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47])
      : "r"(taddr), "r"(taddr + 32u)
      : "memory");
#pragma unroll
  for (int i = 48; i < 64; ++i) r[i] = 0u;
}

// columns [0, 32); the rest of r reads as zero
__device__ __forceinline__ void tmem_ld64_x32(uint32_t taddr, uint32_t (&r)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 32; i < 64; ++i) r[i] = 0u;
}

// columns [0, 16); the rest of r reads as zero
__device__ __forceinline__ void tmem_ld64_x16(uint32_t taddr, uint32_t (&r)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 16; i < 64; ++i) r[i] = 0u;
}

// columns [0, min(n, 64)) of this thread's lane, n a positive multiple of 16
// and the same in the whole warp; columns from n on read as zero
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, int n, uint32_t (&r)[64]) {
  if (n >= 64)
    tmem_ld64_x64(taddr, r);
  else if (n == 48)
    tmem_ld64_x48(taddr, r);
  else if (n == 32)
    tmem_ld64_x32(taddr, r);
  else
    tmem_ld64_x16(taddr, r);
}

// shared-memory descriptor of a K-major, 128-byte-swizzled tile
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3FFFFu) >> 4);  // start address
  d |= uint64_t(1) << 16;                  // leading byte offset (unused for swizzled K-major)
  d |= uint64_t(1024 >> 4) << 32;          // stride byte offset: 8-row groups are 1024 B apart
  d |= uint64_t(1) << 46;                  // descriptor version of tcgen05
  d |= uint64_t(2) << 61;                  // 128-byte swizzle
  return d;
}

// instruction descriptor: bf16 x bf16 -> f32, both operands K-major
__device__ __forceinline__ uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(m >> 4) << 24);
}

__device__ __forceinline__ double dot64(const float* __restrict__ a, const float* __restrict__ x, int d) {
  double s = 0.0;
  for (int i = 0; i < d; ++i) s = __dadd_rn(s, __dmul_rn(double(a[i]), double(x[i])));
  return s;
}

struct Tile {
  int seg;      // segment index
  int first;    // first tile of its segment
  int last;     // last tile of its segment
  int fn;       // CP function index within the repetition
  int sub;      // CP: N tile of the function (its rows start at 128 * sub)
  int fn_last;  // CP: last N tile of the function
  int64_t row0; // first hash row
  int rows;     // N
};

__device__ __forceinline__ Tile tile_of(const HashArgs& A, int seg, int f) {
  Tile t;
  t.seg = seg;
  t.fn = 0;
  t.sub = 0;
  t.fn_last = 1;
  if (seg < A.seg_tables) {
    if (A.family == PF_CROSSPOLYTOPE) {
      t.fn = f / A.nsub;
      t.sub = f - t.fn * A.nsub;
      t.row0 = (int64_t(seg) * A.fns + t.fn) * A.d_pad + int64_t(kBN) * t.sub;
      t.rows = min(kBN, A.d_pad - kBN * t.sub);
      t.first = f == 0;
      t.last = f == A.fns * A.nsub - 1;
      t.fn_last = t.sub == A.nsub - 1;
    } else {
      t.row0 = int64_t(seg) * 128;
      t.rows = 128;
      t.first = t.last = 1;
    }
  } else {
    t.row0 = int64_t(A.L) * A.rows_table + int64_t(seg - A.seg_tables) * 128;
    t.rows = 128;
    t.first = t.last = 1;
  }
  return t;
}

// A run of consecutive segments of one group of P point tiles (P*grp, ...,
// P*grp + P - 1) within the CTA's units.
struct Chunk {
  int pair, seg0, seg1;
};

// The CTA's work, in two phases.  While at least one group of point tiles per
// CTA is left, CTA b takes whole groups b, b + G, b + 2G, ... (G = grid), each
// with all its segments in order: the CTAs then walk the segments in step, so
// each hash-row tile is read from DRAM about once per round of G groups and
// served from L2 to the others, however large the rows are (a bigger index
// than L2 holds would otherwise be re-read from DRAM for every group).  The
// units (group, segment) of the last groups are then split into equal
// contiguous ranges, one per CTA.
struct Sched {
  int64_t rr, rr_end;  // round-robin groups still to take: rr, rr + G, ... < rr_end
  int64_t u, hi;       // then the units [u, hi) of the last groups
};

__device__ __forceinline__ Sched make_sched(const HashArgs& A) {
  const int64_t G = gridDim.x, b = blockIdx.x;
  const int64_t groups = A.units / A.segs;
  const int64_t full = groups / G * G;  // groups taken whole, round robin
  const int64_t tail = (groups - full) * A.segs;
  Sched s;
  s.rr = b;
  s.rr_end = full;
  s.u = full * A.segs + b * tail / G;
  s.hi = full * A.segs + (b + 1) * tail / G;
  return s;
}

__device__ __forceinline__ bool next_chunk(const HashArgs& A, Sched& s, Chunk& c) {
  if (s.rr < s.rr_end) {
    c.pair = int(s.rr);
    c.seg0 = 0;
    c.seg1 = A.segs;
    s.rr += gridDim.x;
    return true;
  }
  if (s.u >= s.hi) return false;
  c.pair = int(s.u / A.segs);
  c.seg0 = int(s.u - int64_t(c.pair) * A.segs);
  c.seg1 = int(min(s.hi - int64_t(c.pair) * A.segs, int64_t(A.segs)));
  s.u = int64_t(c.pair) * A.segs + c.seg1;
  return true;
}

__device__ __forceinline__ int tiles_in_seg(const HashArgs& A, int seg) {
  return (seg < A.seg_tables && A.family == PF_CROSSPOLYTOPE) ? A.fns * A.nsub : 1;
}

struct EpiState {
  uint32_t code;
  uint64_t r0, r1, r2;  // CP over several N tiles: the three largest wide keys of the function so far
};

// float64 projections of up to 4 CP hyperplanes (rows c[q] of function wf,
// those with use[q]) onto x, in index order; chains interleaved for ILP
__device__ __forceinline__ void dot64x4(const float* __restrict__ wf, const int (&c)[4], const bool (&use)[4],
                                        const float* __restrict__ x, int d, int d_pad, double (&out)[4]) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  const float* w0 = wf + int64_t(c[0]) * d_pad;
  const float* w1 = wf + int64_t(c[1]) * d_pad;
  const float* w2 = wf + int64_t(c[2]) * d_pad;
  const float* w3 = wf + int64_t(c[3]) * d_pad;
  for (int i = 0; i < d; ++i) {
    const double xi = double(x[i]);
    if (use[0]) s0 = __dadd_rn(s0, __dmul_rn(double(w0[i]), xi));
    if (use[1]) s1 = __dadd_rn(s1, __dmul_rn(double(w1[i]), xi));
    if (use[2]) s2 = __dadd_rn(s2, __dmul_rn(double(w2[i]), xi));
    if (use[3]) s3 = __dadd_rn(s3, __dmul_rn(double(w3[i]), xi));
  }
  out[0] = s0;
  out[1] = s1;
  out[2] = s2;
  out[3] = s3;
}

// Sort key of the projection v on hyperplane c (c < 128) of a CP function:
// bits 31..8 are |v| cut to its 8 exponent and 16 high mantissa bits, bits
// 7..1 hold 127 - c and bit 0 the sign of v.  Unsigned order of keys is the
// order of |v| up to the cut (less than 2^-16 |v|), ties to the smaller c.
__device__ __forceinline__ uint32_t cp_key(uint32_t vbits, int c) {
  const uint32_t r = __funnelshift_l(vbits, vbits, 1);  // |v| << 1 | sign
  return (r | 0xFEu) - 2u * uint32_t(c);
}
__device__ __forceinline__ float cp_key_abs(uint32_t k) { return __uint_as_float((k >> 1) & 0x7FFFFF80u); }
__device__ __forceinline__ int cp_key_col(uint32_t k) { return 127 - int((k >> 1) & 0x7Fu); }

// the three largest keys seen (m0 > m1 > m2; keys of distinct columns differ)
template <typename K>
__device__ __forceinline__ void top3_push(K k, K& m0, K& m1, K& m2) {
  m2 = max(m2, min(m1, k));
  m1 = max(m1, min(m0, k));
  m0 = max(m0, k);
}

// Wide key of a CP function with several N tiles: the 32-bit key k of column
// c of the tile whose rows start at col0 becomes (the same cut |v|, then
// 1023 - (col0 + c), then the sign), so that keys of different tiles order as
// the 32-bit keys of one tile do (larger |v| first, ties to the smaller row).
__device__ __forceinline__ uint64_t cp_wide_key(uint32_t k, int col0) {
  const uint32_t col = uint32_t(col0 + cp_key_col(k));
  return (uint64_t(k >> 8) << 11) | (uint64_t(1023u - col) << 1) | uint64_t(k & 1u);
}
__device__ __forceinline__ float cp_wide_abs(uint64_t k) { return __uint_as_float(uint32_t(k >> 11) << 7); }
__device__ __forceinline__ int cp_wide_col(uint64_t k) { return 1023 - int((k >> 1) & 1023u); }

// Reserve `cnt` consecutive entries of this CTA's region of the request queue
// for this lane (warp-aggregated: one shared-memory atomic per warp) and
// return the first, counted from the region's start.  Entries at or beyond
// rq_per do not exist: the caller rechecks those inline, so every entry below
// min(count, rq_per) is written by exactly one lane.  All lanes of the warp
// must call it.
__device__ __forceinline__ uint32_t reserve_requests(const HashArgs& A, uint32_t* s_count, uint32_t cnt) {
  const int lane = threadIdx.x & 31;
  uint32_t inc = cnt;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += v;
  }
  const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
  if (total == 0 || !A.rq) return 0xffffffffu;
  uint32_t base = 0;
  if (lane == 0) base = atomicAdd(s_count, total);
  base = __shfl_sync(0xffffffffu, base, 0);
  return base + inc - cnt;
}

__device__ __forceinline__ RecheckReq* request_at(const HashArgs& A, uint32_t local) {
  return A.rq + size_t(blockIdx.x) * A.rq_per + local;
}

// Epilogue of one N tile for the thread's point p (accumulator columns at taddr).
// WIDE: the kernel for d_pad > 128, whose CP functions may span several N
// tiles (with d_pad <= 128 every function is one tile: nsub == 1).
template <bool WIDE>
__device__ __forceinline__ void epilogue(const HashArgs& A, const Tile& t, uint32_t taddr, int64_t p,
                                         EpiState& st, uint32_t* s_count) {
  const bool live = p < A.npts;
  const float* xrow = A.x32 + (live ? p : 0) * A.d_pad;
  if (t.seg < A.seg_tables && A.family == PF_CROSSPOLYTOPE) {
    if (t.first) st.code = 0;
    const float band = A.thr[t.row0];  // one band for all rows of a function
    // the three largest |v| over the function's rows, four independent
    // chains (merged across the N tiles of a function of more than 128 rows);
    // rows c >= d of a function are zero and reach the top three only when
    // fewer than three rows are nonzero (then every row is rechecked)
    uint32_t m0[4] = {0u, 0u, 0u, 0u}, m1[4] = {0u, 0u, 0u, 0u}, m2[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (64 * h < t.rows) {
        uint32_t r[64];
        tmem_ld64(taddr + uint32_t(64 * h), t.rows - 64 * h, r);
#pragma unroll
        for (int i = 0; i < 64; ++i) top3_push(cp_key(r[i], 64 * h + i), m0[i & 3], m1[i & 3], m2[i & 3]);
      }
    }
    uint32_t k0 = m0[0], k1 = m1[0], k2 = m2[0];
#pragma unroll
    for (int q = 1; q < 4; ++q) {
      top3_push(m0[q], k0, k1, k2);
      top3_push(m1[q], k0, k1, k2);
      top3_push(m2[q], k0, k1, k2);
    }
    float a0, a1, a2;
    int arg, cs1;
    bool neg;
    if (!WIDE || A.nsub == 1) {
      a0 = cp_key_abs(k0);
      a1 = cp_key_abs(k1);
      a2 = cp_key_abs(k2);
      arg = cp_key_col(k0);
      cs1 = cp_key_col(k1);
      neg = (k0 & 1u) != 0u;
    } else {
      // the function's rows span several N tiles: merge this tile's top three
      // into the function's, decide after its last tile (uniform in the warp)
      if (t.sub == 0) st.r0 = st.r1 = st.r2 = 0ull;
      const int col0 = kBN * t.sub;
      top3_push(cp_wide_key(k0, col0), st.r0, st.r1, st.r2);
      top3_push(cp_wide_key(k1, col0), st.r0, st.r1, st.r2);
      top3_push(cp_wide_key(k2, col0), st.r0, st.r1, st.r2);
      if (!t.fn_last) return;
      a0 = cp_wide_abs(st.r0);
      a1 = cp_wide_abs(st.r1);
      a2 = cp_wide_abs(st.r2);
      arg = cp_wide_col(st.r0);
      cs1 = cp_wide_col(st.r1);
      neg = (st.r0 & 1ull) != 0ull;
    }
    // every row whose |v| can be within 2*band of the maximum reaches lim:
    // a0 * 2^-15 covers the cut of the keys
    const float lim = a0 - 2.f * band - a0 * 3.0517578125e-05f;
    const bool need = live && (a1 >= lim || a0 < band);
    if (__any_sync(0xffffffffu, need)) {
      // rare: candidates are the top two, or every row once a third reaches lim
      const bool all = a0 < band || a2 >= lim;
      const int cs0 = arg;
      const uint32_t local = reserve_requests(A, s_count, need ? 1u : 0u);
      if (need && local < A.rq_per) {
        // keep the tensor-core decision now; the fix-up kernel rewrites the field
        RecheckReq q;
        q.p = uint32_t(p);
        q.row0 = uint32_t(t.row0 - int64_t(kBN) * t.sub);  // the function's first row
        q.info = uint32_t(t.seg) | (uint32_t(t.fn) << 20) | (3u << 26) | ((all ? 3u : 0u) << 30);
        q.c[0] = uint16_t(cs0);
        q.c[1] = uint16_t(cs1);
        *request_at(A, local) = q;
      } else if (need) {
        const float* wf = A.w32 + (t.row0 - int64_t(kBN) * t.sub) * A.d_pad;
        double bestabs = -1.0, bestval = 0.0;
        int besti = 0;
        if (all) {
          for (int cc = 0; cc < A.d; cc += 4) {
            const int cs[4] = {cc, min(cc + 1, A.d - 1), min(cc + 2, A.d - 1), min(cc + 3, A.d - 1)};
            const bool us[4] = {true, cc + 1 < A.d, cc + 2 < A.d, cc + 3 < A.d};
            double v64[4];
            dot64x4(wf, cs, us, xrow, A.d, A.d_pad, v64);
            for (int u = 0; u < 4; ++u)
              if (us[u] && fabs(v64[u]) > bestabs) {
                bestabs = fabs(v64[u]);
                bestval = v64[u];
                besti = cs[u];
              }
          }
        } else {
          const int cs[4] = {cs0, cs1, cs1, cs1};
          const bool us[4] = {true, true, false, false};
          double v64[4];
          dot64x4(wf, cs, us, xrow, A.d, A.d_pad, v64);
          for (int u = 0; u < 2; ++u) {
            const double av = fabs(v64[u]);
            if (av > bestabs || (av == bestabs && cs[u] < besti)) {
              bestabs = av;
              bestval = v64[u];
              besti = cs[u];
            }
          }
        }
        arg = besti;
        neg = bestval < 0.0;
      }
    }
    const uint32_t value = ((neg ? 1u : 0u) << (A.ell - 1)) | uint32_t(arg);
    st.code |= value << (32 - A.ell * (t.fn + 1));
    if (t.last && live) A.codes[int64_t(t.seg) * A.cj + p * A.cp] = st.code;
    return;
  }
  // 128 one-bit rows: 4 HP repetitions (32 bits each) or 2 sketches (64 bits each)
  const bool is_sketch = t.seg >= A.seg_tables;
  const int64_t row_end = is_sketch ? A.hash_rows : int64_t(A.L) * A.rows_table;
  uint64_t bits0 = 0ull, bits1 = 0ull;
  for (int cb = 0; cb < 128; cb += 16) {
    float v[16];
    tmem_ld16(taddr + uint32_t(cb), v);
    uint32_t needm = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int c = cb + i;
      const int64_t row = t.row0 + c;
      if (row < row_end && live && fabsf(v[i]) < A.thr[row]) needm |= 1u << i;
      if (v[i] >= 0.f) {
        if (c < 64)
          bits0 |= uint64_t(1) << c;
        else
          bits1 |= uint64_t(1) << (c - 64);
      }
    }
    if (__any_sync(0xffffffffu, needm != 0)) {
      uint32_t local = reserve_requests(A, s_count, __popc(needm));
      while (needm) {
        const int i = __ffs(needm) - 1;
        needm &= needm - 1;
        const int c = cb + i;
        const int64_t row = t.row0 + c;
        if (local < A.rq_per) {
          RecheckReq q;
          q.p = uint32_t(p);
          q.row0 = uint32_t(row);
          if (is_sketch) {
            const int64_t r = row - int64_t(A.L) * A.rows_table;
            q.info = uint32_t(r >> 6) | (uint32_t(r & 63) << 20) | (2u << 30);
          } else {
            q.info = uint32_t(row >> 5) | (uint32_t(row & 31) << 20) | (1u << 30);
          }
          q.c[0] = q.c[1] = 0;
          *request_at(A, local) = q;
          ++local;  // stays >= rq_per (including the "no queue" value) once it gets there
        } else {
          const bool bit = dot64(A.w32 + row * A.d_pad, xrow, A.d) >= 0.0;
          const uint64_t m = uint64_t(1) << (c & 63);
          if (c < 64)
            bits0 = bit ? (bits0 | m) : (bits0 & ~m);
          else
            bits1 = bit ? (bits1 | m) : (bits1 & ~m);
        }
      }
    }
  }
  if (!live) return;
  if (is_sketch) {
    const int m0 = (t.seg - A.seg_tables) * 2;
    if (m0 < A.M) A.sk[int64_t(m0) * A.sm + p * A.sp] = bits0;
    if (m0 + 1 < A.M) A.sk[int64_t(m0 + 1) * A.sm + p * A.sp] = bits1;
  } else {
    const uint32_t w[4] = {uint32_t(bits0), uint32_t(bits0 >> 32), uint32_t(bits1), uint32_t(bits1 >> 32)};
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int j = t.seg * 4 + s;
      // column c of repetition j is function c: the first function is the top bit
      if (j < A.L) A.codes[int64_t(j) * A.cj + p * A.cp] = __brev(w[s]);
    }
  }
}

struct TensorMaps {
  CUtensorMap xh, xl;        // A: [npts][d_pad], box {64, 128}
  CUtensorMap wh_f;          // B, CP function tiles (d_pad <= 128): box {64, d_pad}
  CUtensorMap wh_g;          // B, 128-row groups and full 128-row N tiles: box {64, 128}
  CUtensorMap wh_t;          // B, the last N tile of a CP function of d_pad > 128 rows: box {64, d_pad % 128}
};

template <int P>
__global__ void __launch_bounds__(threads_for(P), 1) hash_tc_kernel(HashArgs A, const __grid_constant__ TensorMaps T) {
  constexpr int kPair = P;
  constexpr int kTmemCols = tmem_cols_for(P);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int KB = A.KB, S = A.stages;
  const uint32_t a_bytes = uint32_t(2 * KB * kTileBytes);      // Xh, Xl of one point tile
  const uint32_t sA = smem_u32(base);                          // [kPair][2 splits][KB] tiles
  const uint32_t sB = sA + uint32_t(kPair) * a_bytes;          // [S] tiles
  __shared__ __align__(8) uint64_t bfull[kMaxStages], bempty[kMaxStages], accfull[2][kPair], accempty[2][kPair],
      afull, aempty;
  __shared__ uint32_t s_count;  // entries reserved in this CTA's region of the request queue
  __shared__ uint32_t tmem_base_slot;
  __shared__ volatile int failed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int u = 0; u < S; ++u) {
      mbar_init(smem_u32(&bfull[u]), 1);
      mbar_init(smem_u32(&bempty[u]), 1);
    }
    for (int b = 0; b < 2; ++b)
      for (int pt = 0; pt < kPair; ++pt) {
        mbar_init(smem_u32(&accfull[b][pt]), 1);
        mbar_init(smem_u32(&accempty[b][pt]), 128);
      }
    mbar_init(smem_u32(&afull), 1);
    mbar_init(smem_u32(&aempty), 1);
    failed = 0;
    s_count = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(&tmem_base_slot), kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    uint32_t stage = 0, items_done = 0;
    Sched sc = make_sched(A);
    Chunk ch;
    while (next_chunk(A, sc, ch)) {
      const int seg0 = ch.seg0, seg1 = ch.seg1;
      if (items_done > 0 && !mbar_wait(smem_u32(&aempty), (items_done - 1) & 1)) { failed = 1; break; }
      mbar_expect_tx(smem_u32(&afull), uint32_t(kPair) * a_bytes);
      for (int pt = 0; pt < kPair; ++pt) {
        const int row = (ch.pair * kPair + pt) * kBM;  // rows beyond the points read as zero
        for (int kb = 0; kb < KB; ++kb) {
          tma_load_2d(sA + pt * a_bytes + uint32_t(kb * kTileBytes), &T.xh, kb * 64, row, smem_u32(&afull));
          tma_load_2d(sA + pt * a_bytes + uint32_t((KB + kb) * kTileBytes), &T.xl, kb * 64, row, smem_u32(&afull));
        }
      }
      ++items_done;
      if (A.hold_b) break;  // the MMA and epilogue roles time out (the A loads above complete)
      bool bad = false;
      for (int seg = seg0; seg < seg1 && !bad; ++seg)
        for (int f = 0; f < tiles_in_seg(A, seg) && !bad; ++f) {
          const Tile t = tile_of(A, seg, f);
          const CUtensorMap* mh = t.rows == kBN ? &T.wh_g : A.nsub == 1 ? &T.wh_f : &T.wh_t;
          for (int kb = 0; kb < KB; ++kb, ++stage) {
            const uint32_t slot = stage % S, round = stage / S;
            if (!mbar_wait(smem_u32(&bempty[slot]), (round & 1) ^ 1)) { bad = true; break; }
            mbar_expect_tx(smem_u32(&bfull[slot]), uint32_t(t.rows * 128));
            tma_load_2d(sB + slot * kTileBytes, mh, kb * 64, int(t.row0), smem_u32(&bfull[slot]));
          }
        }
      if (bad) { failed = 1; break; }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer: both point tiles of the pair from every B stage
    uint32_t stage = 0, items_done = 0, g = 0;
    Sched sc = make_sched(A);
    Chunk ch;
    while (!failed && next_chunk(A, sc, ch)) {
      const int seg0 = ch.seg0, seg1 = ch.seg1;
      if (!mbar_wait(smem_u32(&afull), items_done & 1)) { failed = 1; break; }
      ++items_done;
      tc_fence_after();
      bool bad = false;
      for (int seg = seg0; seg < seg1 && !bad; ++seg)
        for (int f = 0; f < tiles_in_seg(A, seg) && !bad; ++f, ++g) {
          const Tile t = tile_of(A, seg, f);
          const uint32_t b = g & 1;
          for (int pt = 0; pt < kPair && !bad; ++pt)
            if (!mbar_wait(smem_u32(&accempty[b][pt]), ((g >> 1) & 1) ^ 1)) bad = true;
          if (bad) break;
          tc_fence_after();
          const uint32_t idesc = idesc_bf16(kBM, t.rows);
          for (int kb = 0; kb < KB; ++kb, ++stage) {
            const uint32_t slot = stage % S, round = stage / S;
            if (!mbar_wait(smem_u32(&bfull[slot]), round & 1)) { bad = true; break; }
            tc_fence_after();
            const uint32_t bt = sB + slot * kTileBytes;
            for (int pt = 0; pt < kPair; ++pt) {
              const uint32_t d_tmem = tmem + (b * kPair + pt) * kBN;
              // the hyperplane tile is exact in bfloat16: Xh*W and Xl*W
              for (int half = 0; half < 2; ++half) {
                const uint32_t at = sA + pt * a_bytes + uint32_t(((half ? KB : 0) + kb) * kTileBytes);
                for (int kk = 0; kk < 4; ++kk)
                  mma_bf16(d_tmem, sw128_desc(at + kk * 32), sw128_desc(bt + kk * 32), idesc,
                           (kb | half | kk) ? 1u : 0u);
              }
            }
            mma_commit(smem_u32(&bempty[slot]));
          }
          for (int pt = 0; pt < kPair; ++pt) mma_commit(smem_u32(&accfull[b][pt]));
        }
      mma_commit(smem_u32(&aempty));
      if (bad) { failed = 1; break; }
    }
  } else if (warp >= 2) {
    // ---------------- epilogue: group pt (warps 2-5: point tile 0, 6-9: point tile 1),
    // thread = point, TMEM lane quarter = warp % 4 (the only quarter a warp may read)
    const int pt = (warp - 2) >> 2, quarter = warp & 3;
    uint32_t g = 0;
    Sched sc = make_sched(A);
    Chunk ch;
    while (!failed && next_chunk(A, sc, ch)) {
      const int seg0 = ch.seg0, seg1 = ch.seg1;
      const int64_t p = int64_t(ch.pair * kPair + pt) * kBM + quarter * 32 + lane;
      EpiState st;
      st.code = 0;
      bool bad = false;
      for (int seg = seg0; seg < seg1 && !bad; ++seg)
        for (int f = 0; f < tiles_in_seg(A, seg) && !bad; ++f, ++g) {
          const Tile t = tile_of(A, seg, f);
          const uint32_t b = g & 1;
          if (!mbar_wait(smem_u32(&accfull[b][pt]), (g >> 1) & 1)) { bad = true; break; }
          tc_fence_after();
          epilogue<P == 1>(A, t, tmem + (uint32_t(quarter * 32) << 16) + (b * kPair + pt) * kBN, p, st, &s_count);
          tc_fence_before();
          mbar_arrive(smem_u32(&accempty[b][pt]));
        }
      if (bad) { failed = 1; break; }
    }
  }
  __syncthreads();
  if (tid == 0 && A.rq) A.rq_count[blockIdx.x] = min(s_count, A.rq_per);
  if (failed && tid == 0) atomicOr(A.error, 2);
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

// float64 projections, in index order, of the rows w[u] with bit u of `use`
// onto x (d elements): four elements per load, the loads of the next group
// issued before the arithmetic of this one (rows start 16-byte aligned)
__device__ __forceinline__ void dot64_rows(const float* const (&w)[4], uint32_t use, const float* __restrict__ x,
                                           int d, double (&out)[4]) {
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  const int d4 = d & ~3;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 xv = z, wv[4] = {z, z, z, z};
  if (d4 > 0) {
    xv = __ldg(reinterpret_cast<const float4*>(x));
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (use & (1u << u)) wv[u] = __ldg(reinterpret_cast<const float4*>(w[u]));
  }
  for (int i = 0; i < d4; i += 4) {
    float4 xn = z, wn[4] = {z, z, z, z};
    if (i + 4 < d4) {
      xn = __ldg(reinterpret_cast<const float4*>(x + i + 4));
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (use & (1u << u)) wn[u] = __ldg(reinterpret_cast<const float4*>(w[u] + i + 4));
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (!(use & (1u << u))) continue;
      s[u] = __dadd_rn(s[u], __dmul_rn(double(wv[u].x), double(xv.x)));
      s[u] = __dadd_rn(s[u], __dmul_rn(double(wv[u].y), double(xv.y)));
      s[u] = __dadd_rn(s[u], __dmul_rn(double(wv[u].z), double(xv.z)));
      s[u] = __dadd_rn(s[u], __dmul_rn(double(wv[u].w), double(xv.w)));
    }
    xv = xn;
#pragma unroll
    for (int u = 0; u < 4; ++u) wv[u] = wn[u];
  }
  for (int i = d4; i < d; ++i)
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (use & (1u << u)) s[u] = __dadd_rn(s[u], __dmul_rn(double(w[u][i]), double(x[i])));
#pragma unroll
  for (int u = 0; u < 4; ++u) out[u] = s[u];
}

// float32 projections, in index order by fused multiply-add, of the rows w[u]
// with bit u of `use` onto x, each with a bound on its distance to the float64
// projection in index order: both are within (d+1)*2^-24 * sum|w_i x_i| of the
// exact sum (plus the underflow of d products), so they are within
// err = (d+2)*2^-23 * sum|w_i x_i| + d*2^-126 of each other (the float32 sum of
// |w_i x_i| is itself within a factor 1 + (d+1)*2^-24 of the exact one).
// A decision whose float32 margin exceeds the bound is the float64 decision.
__device__ __forceinline__ void dot32_rows(const float* const (&w)[4], uint32_t use, const float* __restrict__ x,
                                           int d, float (&out)[4], float (&err)[4]) {
  float s[4] = {0.f, 0.f, 0.f, 0.f}, a[4] = {0.f, 0.f, 0.f, 0.f};
  const int d4 = d & ~3;
  for (int i = 0; i < d4; i += 4) {
    const float4 xv = __ldg(reinterpret_cast<const float4*>(x + i));
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (!(use & (1u << u))) continue;
      const float4 wv = __ldg(reinterpret_cast<const float4*>(w[u] + i));
      s[u] = __fmaf_rn(wv.x, xv.x, s[u]);
      s[u] = __fmaf_rn(wv.y, xv.y, s[u]);
      s[u] = __fmaf_rn(wv.z, xv.z, s[u]);
      s[u] = __fmaf_rn(wv.w, xv.w, s[u]);
      a[u] = __fmaf_rn(fabsf(wv.x), fabsf(xv.x), a[u]);
      a[u] = __fmaf_rn(fabsf(wv.y), fabsf(xv.y), a[u]);
      a[u] = __fmaf_rn(fabsf(wv.z), fabsf(xv.z), a[u]);
      a[u] = __fmaf_rn(fabsf(wv.w), fabsf(xv.w), a[u]);
    }
  }
  for (int i = d4; i < d; ++i)
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (use & (1u << u)) {
        s[u] = __fmaf_rn(w[u][i], x[i], s[u]);
        a[u] = __fmaf_rn(fabsf(w[u][i]), fabsf(x[i]), a[u]);
      }
  const float f = float(d + 2) * 1.1920928955078125e-07f;  // (d+2) * 2^-23
  const float tiny = float(d) * 1.1754943508222875e-38f;   // d * 2^-126
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    out[u] = s[u];
    err[u] = __fmaf_ru(f, a[u], tiny);
  }
}

// rewrite the CP field of function fn of repetition j for point p with the
// float64 decision (row besti, sign of bestval)
__device__ __forceinline__ void store_cp_field(const HashArgs& A, uint32_t info, int64_t p, int besti,
                                               double bestval) {
  const int j = int(info & 0xFFFFFu), fn = int((info >> 20) & 63u);
  const uint32_t value = ((bestval < 0.0 ? 1u : 0u) << (A.ell - 1)) | uint32_t(besti);
  const int shift = 32 - A.ell * (fn + 1);
  const uint32_t field = ((1u << A.ell) - 1u) << shift;
  uint32_t* w = A.codes + int64_t(j) * A.cj + p * A.cp;
  atomicAnd(w, ~field);
  atomicOr(w, value << shift);
}

// One request of kind 0 (CP, listed candidate rows), 1 (HP bit) or 2 (sketch bit).
__device__ __forceinline__ void recheck_one(const HashArgs& A, const RecheckReq& q) {
  const int64_t p = q.p;
  const float* xrow = A.x32 + p * A.d_pad;
  const uint32_t kind = q.info >> 30;
  if (kind == 0) {
    const uint32_t use = (q.info >> 26) & 3u;
    const float* wf = A.w32 + int64_t(q.row0) * A.d_pad;
    const int cs[4] = {q.c[0], q.c[1], q.c[1], q.c[1]};
    const float* w[4] = {wf + int64_t(cs[0]) * A.d_pad, wf + int64_t(cs[1]) * A.d_pad, wf + int64_t(cs[2]) * A.d_pad,
                         wf + int64_t(cs[3]) * A.d_pad};
    // float32 first: the row whose |value| exceeds every other listed row's
    // by more than both bounds, with a sign outside its bound, is the
    // float64 decision
    float v32[4], e32[4];
    dot32_rows(w, use, xrow, A.d, v32, e32);
    int top = -1;
    for (int u = 0; u < 4 && top < 0; ++u) {
      if (!(use & (1u << u)) || !(fabsf(v32[u]) > e32[u])) continue;
      bool clear = true;
      for (int o = 0; o < 4; ++o)
        if (o != u && (use & (1u << o)) && !(fabsf(v32[u]) - fabsf(v32[o]) > e32[u] + e32[o])) clear = false;
      if (clear) top = u;
    }
    if (top >= 0) {
      store_cp_field(A, q.info, p, cs[top], double(v32[top]));
      return;
    }
    double v64[4];
    dot64_rows(w, use, xrow, A.d, v64);
    double bestabs = -1.0, bestval = 0.0;
    int besti = 0;
    for (int u = 0; u < 4; ++u) {
      if (!(use & (1u << u))) continue;
      const double av = fabs(v64[u]);
      if (av > bestabs || (av == bestabs && cs[u] < besti)) {
        bestabs = av;
        bestval = v64[u];
        besti = cs[u];
      }
    }
    store_cp_field(A, q.info, p, besti, bestval);
    return;
  }
  const float* w[4] = {A.w32 + int64_t(q.row0) * A.d_pad, xrow, xrow, xrow};
  float v32[4], e32[4];
  dot32_rows(w, 1u, xrow, A.d, v32, e32);
  bool bit;
  if (fabsf(v32[0]) > e32[0]) {
    bit = v32[0] > 0.f;  // the float64 value has the same sign (and is not zero)
  } else {
    double v64[4];
    dot64_rows(w, 1u, xrow, A.d, v64);
    bit = v64[0] >= 0.0;
  }
  const int idx = int(q.info & 0xFFFFFu), b = int((q.info >> 20) & 63u);
  if (kind == 1) {
    uint32_t* cw = A.codes + int64_t(idx) * A.cj + p * A.cp;
    const uint32_t m = 1u << (31 - b);
    if (bit) atomicOr(cw, m); else atomicAnd(cw, ~m);
  } else {
    unsigned long long* sw = reinterpret_cast<unsigned long long*>(A.sk + int64_t(idx) * A.sm + p * A.sp);
    const unsigned long long m = 1ull << b;
    if (bit) atomicOr(sw, m); else atomicAnd(sw, ~m);
  }
}

// One CP request of kind 3 (every row a candidate), by a whole warp: lane l
// takes rows l, l+32, ... (d <= 320, in groups of 128 rows), each in float64
// in index order, then the warp keeps the largest |value|, ties to the
// smaller row.
__device__ __forceinline__ void recheck_all_rows(const HashArgs& A, uint32_t p32, uint32_t row0, uint32_t info) {
  const int lane = threadIdx.x & 31;
  const int64_t p = p32;
  const float* xrow = A.x32 + p * A.d_pad;
  const float* wf = A.w32 + int64_t(row0) * A.d_pad;
  // rows c0 + lane + 32 u (u < 4) of the group at c0
  auto group = [&](int c0, const float* (&w)[4]) {
    uint32_t use = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = c0 + lane + 32 * u;
      w[u] = wf + int64_t(min(c, A.d - 1)) * A.d_pad;
      if (c < A.d) use |= 1u << u;
    }
    return use;
  };
  // float32 first: decided if the largest |value| exceeds every other row's by
  // more than the largest bound twice over and its sign is outside the bound
  {
    float m1 = -1.f, m2 = -1.f, emax = 0.f, val = 0.f;
    int i1 = 0;
    for (int c0 = 0; c0 < A.d; c0 += 128) {
      const float* w[4];
      const uint32_t use = group(c0, w);
      float v32[4], e32[4];
      dot32_rows(w, use, xrow, A.d, v32, e32);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (!(use & (1u << u))) continue;
        const float av = fabsf(v32[u]);
        emax = fmaxf(emax, e32[u]);
        if (av > m1) {
          m2 = m1;
          m1 = av;
          i1 = c0 + lane + 32 * u;
          val = v32[u];
        } else {
          m2 = fmaxf(m2, av);
        }
      }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      const float o1 = __shfl_xor_sync(0xffffffffu, m1, off), o2 = __shfl_xor_sync(0xffffffffu, m2, off);
      const float oe = __shfl_xor_sync(0xffffffffu, emax, off), ov = __shfl_xor_sync(0xffffffffu, val, off);
      const int oi = __shfl_xor_sync(0xffffffffu, i1, off);
      emax = fmaxf(emax, oe);
      if (o1 > m1 || (o1 == m1 && oi < i1)) {
        m2 = fmaxf(m1, o2);
        m1 = o1;
        i1 = oi;
        val = ov;
      } else {
        m2 = fmaxf(m2, o1);
      }
    }
    if (m1 > emax && m1 - m2 > 2.f * emax) {
      if (lane == 0) store_cp_field(A, info, p, i1, double(val));
      return;
    }
  }
  double bestabs = -1.0, bestval = 0.0;
  int besti = 0x7FFFFFFF;
  for (int c0 = 0; c0 < A.d; c0 += 128) {  // rows visited in increasing order: the first of equals stays
    const float* w[4];
    const uint32_t use = group(c0, w);
    double v64[4];
    dot64_rows(w, use, xrow, A.d, v64);
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if ((use & (1u << u)) && fabs(v64[u]) > bestabs) {
        bestabs = fabs(v64[u]);
        bestval = v64[u];
        besti = c0 + lane + 32 * u;
      }
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const double oa = __shfl_xor_sync(0xffffffffu, bestabs, off);
    const double ov = __shfl_xor_sync(0xffffffffu, bestval, off);
    const int oi = __shfl_xor_sync(0xffffffffu, besti, off);
    if (oa > bestabs || (oa == bestabs && oi < besti)) {
      bestabs = oa;
      bestval = ov;
      besti = oi;
    }
  }
  if (lane == 0) store_cp_field(A, info, p, besti, bestval);
}

// Deferred float64 rechecks: `blocks_per_region` CTAs per region of the queue;
// a warp takes 32 consecutive requests, one per lane, and then does the
// "all rows" requests among them together.  Each request rewrites the decided
// field of a code (CP function value or HP bit) or sketch bit with the float64
// decision.  Fields of different requests are disjoint, so the two atomic
// updates (clear, then set) of concurrent requests on one word commute.
__global__ void recheck_kernel(HashArgs A, int blocks_per_region) {
  const int region = blockIdx.x / blocks_per_region, sub = blockIdx.x % blocks_per_region;
  const uint32_t count = min(A.rq_count[region], A.rq_per);
  const RecheckReq* rq = A.rq + size_t(region) * A.rq_per;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t stride = uint32_t(blocks_per_region) * blockDim.x;
  for (uint32_t base = uint32_t(sub) * blockDim.x + uint32_t(warp) * 32u; base < count; base += stride) {
    const uint32_t i = base + uint32_t(lane);
    const bool has = i < count;
    RecheckReq q;
    q.p = q.row0 = q.info = 0u;
    q.c[0] = q.c[1] = 0;
    if (has) q = rq[i];
    const bool full = has && (q.info >> 30) == 3u;
    if (has && !full) recheck_one(A, q);
    uint32_t fm = __ballot_sync(0xffffffffu, full);
    while (fm) {
      const int src = __ffs(fm) - 1;
      fm &= fm - 1;
      const uint32_t p = __shfl_sync(0xffffffffu, q.p, src);
      const uint32_t row0 = __shfl_sync(0xffffffffu, q.row0, src);
      const uint32_t info = __shfl_sync(0xffffffffu, q.info, src);
      recheck_all_rows(A, p, row0, info);
    }
  }
}

}  // namespace

uint32_t recheck_capacity(const pf_index* ix, int64_t npts, int tables) {
  const int64_t per_table = ix->family == PF_SIMHASH ? ix->lay.Kb : ix->lay.fns;
  const int64_t per = std::max<int64_t>(48, (int64_t(tables) * per_table + 19) / 20 + (64 * int64_t(ix->M) + 255) / 256);
  return uint32_t(std::min<int64_t>(npts * per + 65536, 0xFFFFFFFFll));
}

int hash_tc_stages(int d_pad) {
  const int KB = (d_pad + 63) / 64;
  // the static barriers (padded to 1 KB) and the 1 KB alignment slack
  const int left = kSmemLimit - 2048 - pair_for(d_pad) * 2 * KB * kTileBytes;
  return std::min(kMaxStages, left / kTileBytes);
}

size_t hash_tc_smem(int d_pad) {
  const int KB = (d_pad + 63) / 64;
  return size_t(pair_for(d_pad) * 2 * KB + hash_tc_stages(d_pad)) * kTileBytes + 1024;
}

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

// 2-D bf16 tensor [rows][d_pad] (row-major), box {64, box_rows}, 128-byte swizzle;
// rows and columns outside the tensor read as zero
bool make_map(CUtensorMap* m, const void* base, int64_t rows, int d_pad, int box_rows) {
  EncodeTiled enc = encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {cuuint64_t(d_pad), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(d_pad) * 2};
  const cuuint32_t box[2] = {64u, cuuint32_t(box_rows)};
  const cuuint32_t estr[2] = {1u, 1u};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t launch_hash_tc(const pf_index* ix, const __nv_bfloat16* xh, const __nv_bfloat16* xl, const float* x32,
                           int64_t npts, uint32_t* codes, int64_t cj, int64_t cp, uint64_t* sk, int64_t sm,
                           int64_t sp, int32_t* error, RecheckReq* rq, uint32_t* rq_count, uint32_t rq_cap,
                           cudaStream_t s, int tables) {
  if (npts <= 0) return cudaSuccess;
  HashArgs A;
  A.xh = xh;
  A.xl = xl;
  A.x32 = x32;
  A.npts = npts;
  A.wh = ix->Whi;
  A.w32 = ix->W32;
  A.thr = ix->Wthr;
  A.hash_rows = ix->hash_rows;
  A.d = ix->d;
  A.d_pad = ix->lay.d_pad;
  A.KB = (A.d_pad + 63) / 64;
  A.family = ix->family;
  A.L = tables;
  A.M = ix->M;
  A.fns = ix->lay.fns;
  A.ell = ix->lay.ell;
  A.rows_table = ix->lay.rows_table;
  A.nsub = ix->family == PF_CROSSPOLYTOPE ? (A.d_pad + kBN - 1) / kBN : 1;
  A.seg_tables = ix->family == PF_CROSSPOLYTOPE ? tables : (tables + 3) / 4;
  A.segs = A.seg_tables + (ix->M + 1) / 2;
  const int P = pair_for(A.d_pad);
  const int64_t mtiles = (npts + kBM - 1) / kBM;
  A.units = (mtiles + P - 1) / P * A.segs;
  A.stages = hash_tc_stages(A.d_pad);
  A.hold_b = ix->hold_weight_loads;
  A.codes = codes;
  A.cj = cj;
  A.cp = cp;
  A.sk = sk;
  A.sm = sm;
  A.sp = sp;
  A.error = error;
  const int grid = int(std::min<int64_t>(A.units, ix->num_sms));
  A.rq = rq_cap && rq_count ? rq : nullptr;
  A.rq_count = rq_count;
  A.rq_per = A.rq ? rq_cap / uint32_t(grid) : 0u;
  TensorMaps T;
  // B boxes: a whole CP function (d_pad <= 128), a 128-row group or N tile,
  // and the last N tile of a function of more rows (unused maps repeat wh_g)
  const int fn_rows = ix->family == PF_CROSSPOLYTOPE && A.nsub == 1 ? A.d_pad : kBN;
  const int tail_rows = ix->family == PF_CROSSPOLYTOPE && A.d_pad % kBN != 0 && A.nsub > 1 ? A.d_pad % kBN : kBN;
  if (!make_map(&T.xh, xh, npts, A.d_pad, kBM) || !make_map(&T.xl, xl, npts, A.d_pad, kBM) ||
      !make_map(&T.wh_f, ix->Whi, ix->hash_rows, A.d_pad, fn_rows) ||
      !make_map(&T.wh_g, ix->Whi, ix->hash_rows, A.d_pad, kBN) ||
      !make_map(&T.wh_t, ix->Whi, ix->hash_rows, A.d_pad, tail_rows))
    return cudaErrorInvalidValue;
  const size_t smem = hash_tc_smem(A.d_pad);
  void (*kern)(HashArgs, TensorMaps) = P == 2 ? hash_tc_kernel<2> : hash_tc_kernel<1>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  kern<<<grid, threads_for(P), smem, s>>>(A, T);
  e = cudaGetLastError();
  if (e != cudaSuccess || !A.rq) return e;
  recheck_kernel<<<4 * grid, 256, 0, s>>>(A, 4);
  return cudaGetLastError();
}

}  // namespace pf
