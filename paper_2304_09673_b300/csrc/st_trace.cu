// st_trace.cu -- synchronized sphere tracing of screen tiles (Sec. 8,
// Algorithm 2) over pruned tree views built by the sparse bottom-up traversal
// (Sec. 7, Algorithm 1, with the usage bits of Sec. 9) and evaluated by
// Algorithm 3.
//
// Execution model (own design for sm_103a):
//   * persistent CTAs of kWarps warps, three per SM; a CTA traces one tile at
//     a time, tiles handed out longest A-buffer list first from a global
//     counter (one launch can cover the tiles of many scenes); once every
//     tile has been handed out, a tile still tracing after a cycle budget
//     shares its pending rays with CTAs out of work (split records, below);
//   * warp 0 walks the tile's depth-sorted A-buffer list, segmenting the tile
//     frustum into subfrustums [z_begin, z_end] with a fixed active primitive
//     set (Sec. 8 "tracking active primitives"; discard, fetch and sorted
//     merge are warp-parallel), builds the pruned view of subfrustum k + 1
//     (lowest common ancestors of consecutive active primitives, the same
//     view as Algorithm 1) and fills its shared parameter cache while all
//     warps march subfrustum k;
//   * each warp sphere-traces up to two rays per lane in lockstep over the
//     same view (warp-uniform node sequence, no divergence in the
//     interpreter); a lane whose ray hits, leaves the subfrustum or reaches
//     the step cap takes the next pending ray of the tile; with few rays left
//     a warp compacts them to one evaluation chain per lane, then evaluates
//     each remaining ray with the whole warp (tail mode) and hands rays to
//     idle warps of the tile;
//   * step modes: plain f / (L |d|); fixed or learned over-relaxation, every
//     relaxed step verified by the sphere-overlap test (Sec. 10); recording
//     of plain steps for training;
//   * hits are refined with Newton steps on the ray (dual numbers) and get
//     the normalised forward-mode gradient of f_A as normal.
#include <cstdint>
#include <type_traits>

#include "st_field.cuh"
#include "st_geom.cuh"
#include "st_kernels.h"
#include "st_mlp.cuh"

namespace st {

constexpr int kWarps = 4;   // warps per CTA; a CTA traces one tile at a time
constexpr int kFurtherBit = 64;   // instance bit: the interpreter evaluates the further families
constexpr int kAllFamBit = 256;   // instance bit (with kFurtherBit): ... including the rounded triangle and quadric
constexpr int kStagedBit = 128;   // instance bit: views in global memory, evaluated in staged chunks
// instance bit (staged launches with the large parameter cache, whose shared
// memory allows two CTAs per SM anyway): registers for two CTAs per SM
// instead of three (measured on B300, 10k clustered 1920x1080: 7-9 % faster)
constexpr int kWideBit = 512;
// instance bit (staged launches with cta_min_view > 0): the CTA-split
// evaluation is compiled in (its code costs the lockstep loop of a staged
// instance ~15 % when it is present, measured on B300, so launches without
// the split use instances without it)
constexpr int kCtaBit = 1024;
constexpr int kStageWords = 64;   // float4 record words of a warp's stage buffer (staged instances)
constexpr int kTileStatWords = 24;   // words per tile of the optional diagnostics
constexpr int kR = 2;       // rays per lane (shared node decode, two evaluation chains)
// CTA-split evaluation (staged instances): once a subfrustum with a large view
// is down to kCtaMaxRays rays, one warp holds them all and each warp evaluates
// a quarter of the view for them (see build_cta_split and march_sub).
constexpr int kCtaMaxRays = 64;     // rays of the owner warp (two per lane)
constexpr int kCtaTopMax = 256;     // words of a view's top program
constexpr int kCtaOutMax = 128;     // output slots of the segments (one float2 per lane each)
constexpr int kCtaDone = 2;         // owner -> helpers: the subfrustum is finished
constexpr int kMaxTileRaysCta = 1024 / kWarps;   // owner's share of a 32x32 tile's hits at most
// Tail queue entries: every ray once through tail sharing, and on launches
// with the CTA split the rays that helpers hand to the owner.
__host__ __device__ inline int tq_cap(const TraceLaunch &L) {
  return L.max_tile_rays + (L.cta_min_view > 0 ? kCtaMaxRays : 0);
}

int trace_warps_per_cta() { return kWarps; }

enum RayStatus : uint32_t { R_ALIVE = 0, R_HIT = 1, R_UNCONV = 2 };
// ray_st keeps a ray's step count in its low 24 bits: the step cap of the
// modes without one.
constexpr int kStepFieldMax = 0xFFFFFF;

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
// View-build stacks: value stack (uint2) and pending-operator stack (uint4),
// stack_slots + 2 entries each.
__host__ __device__ inline size_t bstk_words(const TraceLaunch &L) { return 6 * (size_t)(L.stack_slots + 2); }

// Shared memory of a CTA: ray state, two pending-ray lists, per-warp hit
// lists, per-warp evaluation stacks (float2 slots), the Algorithm 1 stack,
// and (when they fit) the active set and two pruned views.
__host__ __device__ inline size_t smem_fixed_bytes(const TraceLaunch &L) {
  const size_t r = (size_t)L.max_tile_rays;
  return align16(r * 4) + align16(r * 4) + 2 * align16(r * 2) + (size_t)kWarps * align16(r * 2) +
         align16(r * 16) + align16(r * 8) + align16((size_t)tq_cap(L) * 8) +
         (size_t)kWarps * align16((size_t)L.stack_slots * 32 * 8) + align16(bstk_words(L) * 4) +
         2 * (size_t)L.dc_words * 16 + (L.mlp ? kMlpPackBytes : 0) +
         (L.staged ? (size_t)kWarps * kStageWords * 16 : 0);
}
constexpr int kMaxLevels = 64;   // operator levels of a view usable by the tail mode

// CTA-split areas of a work area: two segment streams, two top programs, the
// top programs' operator records, the segments' output slots and the owner's
// points (global memory: shared memory has no room left on these launches),
// and the split's build scratch (parent, left child, flags, slot per node).
constexpr int kCtaPtsWords = 3 * 32 / 2;   // float4 words of the owner's points (x, y, z pairs per lane)
__host__ __device__ inline size_t cta_bytes(const TraceLaunch &L) {
  if (L.cta_min_view <= 0) return 0;
  const size_t v = (size_t)L.view_cap;
  return 2 * align16((v + kCtaOutMax) * 4) + 2 * align16((size_t)kCtaTopMax * 4) +
         (size_t)(2 * kCtaTopMax + 16 * kCtaOutMax + kCtaPtsWords) * 16 + 4 * align16(v * 4);
}
__host__ __device__ inline size_t work_bytes(const TraceLaunch &L) {
  return align16((size_t)L.act_cap * 4) * 4 + 2 * align16((size_t)L.view_cap * 4) +
         2 * align16((size_t)L.act_cap * 8) + 2 * align16((size_t)(kMaxLevels + 1) * 4) +
         align16((size_t)L.act_cap * 8) + cta_bytes(L);
}
__host__ __device__ inline size_t smem_per_cta(const TraceLaunch &L) {
  return smem_fixed_bytes(L) + (L.work_in_smem ? work_bytes(L) : 0);
}
size_t trace_smem_per_warp(const TraceLaunch &L) { return smem_per_cta(L) / kWarps; }
uint32_t trace_work_words(const TraceLaunch &L) { return (uint32_t)(work_bytes(L) / 4); }

// The larger cache (2032 float4 words, twice) holds the parameters of views
// of ~600 primitives but leaves room for two CTAs per SM instead of three
// (2032 rather than 2048: two CTAs with the CTA split's tail-queue entries
// and shared protocol words still fit the SM's 228 KB).
// That pays when the launch is bound by its heaviest tiles, whose long lists
// make large views and many subfrustums (their warps then get a larger share
// of the SM), not when the work is spread over many more tiles than CTAs:
// measured on B300, 10k clustered primitives at 1920x1080 gain 4-10 %
// (5k: 22 %) and at 3840x2160 lose 25-40 %.  The test compares the longest
// list with the entries per CTA.
int trace_dcache_words(int view_cap, uint32_t max_overlap, uint64_t n_entries, int n_sm) {
  if (view_cap <= 2048) return 640;
  const double per_cta = (double)n_entries / (3.0 * std::max(n_sm, 1));
  return (double)max_overlap > 0.3 * per_cta ? 2032 : 640;
}

struct CtaWork {
  float *ray_z;       // [rays] depth reached by each ray
  uint32_t *ray_st;   // [rays] steps | status << 24
  uint16_t *alive[2]; // pending rays, read list / append list (alternating)
  uint16_t *hits;     // [kWarps][rays] rays that hit in the current subfrustum
  float4 *rs4;        // [rays] state of a ray handed to another warp: rp, dzp, zf, zs
  float2 *rs2;        // [rays] ... rs, f at the previous point
  unsigned long long *tq;  // [rays] shared tail queue: (tag << 32) | ray
  float2 *stk;        // [kWarps][stack_slots][32]
  uint32_t *bstk;     // Algorithm 1 stack
  uint32_t *act[2];
  float *act_ze[2];
  uint32_t *view[2];
  float4 *dc[2];       // shared parameter cache of each view (the paper's D_cache)
  unsigned char *mlp;  // packed MLP weights (learned step) or null
  float4 *stage;       // [kWarps][kStageWords] record stages (views in global memory) or null
  uint2 *ops[2];       // operators of each view sorted by level: (self | left << 16, right)
  int *lvl_off[2];     // [kMaxLevels + 1] level offsets into ops
  uint2 *sort_tmp;     // view build: level-sort scratch [act_cap]
  uint32_t *cseg[2];   // CTA split of each view: the four segment streams
  uint32_t *ctop[2];   // ... the top program
  float4 *crec;        // [2 kCtaTopMax] top programs' operator records, then
                       // [kCtaOutMax][32] float2 output slots of the segments,
                       // then [3][32] float2 points of the owner's pass
  uint32_t *cscr;      // [4][view_cap] split build scratch
};

__device__ CtaWork carve(unsigned char *p, const TraceLaunch &L, uint32_t *gwork) {
  CtaWork w;
  const size_t r = (size_t)L.max_tile_rays;
  w.ray_z = (float *)p; p += align16(r * 4);
  w.ray_st = (uint32_t *)p; p += align16(r * 4);
  w.alive[0] = (uint16_t *)p; p += align16(r * 2);
  w.alive[1] = (uint16_t *)p; p += align16(r * 2);
  w.hits = (uint16_t *)p; p += (size_t)kWarps * align16(r * 2);
  w.rs4 = (float4 *)p; p += align16(r * 16);
  w.rs2 = (float2 *)p; p += align16(r * 8);
  w.tq = (unsigned long long *)p; p += align16((size_t)tq_cap(L) * 8);
  w.stk = (float2 *)p; p += (size_t)kWarps * align16((size_t)L.stack_slots * 32 * 8);
  w.bstk = (uint32_t *)p; p += align16(bstk_words(L) * 4);
  w.dc[0] = (float4 *)p; p += (size_t)L.dc_words * 16;
  w.dc[1] = (float4 *)p; p += (size_t)L.dc_words * 16;
  w.mlp = nullptr;
  if (L.mlp) { w.mlp = p; p += kMlpPackBytes; }
  w.stage = nullptr;
  if (L.staged) { w.stage = (float4 *)p; p += (size_t)kWarps * kStageWords * 16; }
  unsigned char *q = L.work_in_smem ? p : (unsigned char *)gwork;
  const size_t a = align16((size_t)L.act_cap * 4);
  w.act[0] = (uint32_t *)q; q += a;
  w.act[1] = (uint32_t *)q; q += a;
  w.act_ze[0] = (float *)q; q += a;
  w.act_ze[1] = (float *)q; q += a;
  w.view[0] = (uint32_t *)q; q += align16((size_t)L.view_cap * 4);
  w.view[1] = (uint32_t *)q; q += align16((size_t)L.view_cap * 4);
  w.ops[0] = (uint2 *)q; q += align16((size_t)L.act_cap * 8);
  w.ops[1] = (uint2 *)q; q += align16((size_t)L.act_cap * 8);
  w.lvl_off[0] = (int *)q; q += align16((size_t)(kMaxLevels + 1) * 4);
  w.lvl_off[1] = (int *)q; q += align16((size_t)(kMaxLevels + 1) * 4);
  w.sort_tmp = (uint2 *)q; q += align16((size_t)L.act_cap * 8);
  w.cseg[0] = w.cseg[1] = w.ctop[0] = w.ctop[1] = w.cscr = nullptr;
  w.crec = nullptr;
  if (L.cta_min_view > 0) {
    const size_t v = (size_t)L.view_cap;
    w.cseg[0] = (uint32_t *)q; q += align16((v + kCtaOutMax) * 4);
    w.cseg[1] = (uint32_t *)q; q += align16((v + kCtaOutMax) * 4);
    w.ctop[0] = (uint32_t *)q; q += align16((size_t)kCtaTopMax * 4);
    w.ctop[1] = (uint32_t *)q; q += align16((size_t)kCtaTopMax * 4);
    w.crec = (float4 *)q; q += (size_t)(2 * kCtaTopMax + 16 * kCtaOutMax + kCtaPtsWords) * 16;
    w.cscr = (uint32_t *)q;
  }
  return w;
}

// Select one of a pair of buffers by a run-time bit without indexing an
// array (keeps the work-area pointers in registers).
template <class P>
__device__ __forceinline__ P pick(P const (&a)[2], int i) { return (i & 1) ? a[1] : a[0]; }

__device__ __forceinline__ int find_job_tile(const Job *jobs, int n_jobs, uint32_t item) {
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].tile_base <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Position of the k-th (0-based) set bit of m (k < popc(m)).
// Named barrier over all warps of the CTA (ids 1 and 2; 0 is __syncthreads).
__device__ __forceinline__ void cta_bar(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kWarps * 32) : "memory");
}

__device__ __forceinline__ int kth_set_bit(uint32_t m, int k) {
  int pos = 0;
#pragma unroll
  for (int b = 16; b >= 1; b >>= 1) {
    const uint32_t low = pos + b >= 32 ? m : (m & ((1u << (pos + b)) - 1u));
    if (__popc(low) <= k) pos += b;
  }
  return pos;
}

// Number of lanes l < n whose value v (sorted ascending over lanes 0..n-1)
// is below q; q may differ per lane.  Five shuffles.
__device__ __forceinline__ int lanes_below(uint32_t v, int n, uint32_t q) {
  int c = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    const int probe = c + step - 1;
    const uint32_t x = __shfl_sync(0xFFFFFFFFu, v, probe & 31);
    if (probe < n && x < q) c += step;
  }
  // the steps reach 31 at most: all 32 below q
  const uint32_t last = __shfl_sync(0xFFFFFFFFu, v, 31);
  if (c == 31 && n == 32 && last < q) c = 32;
  return c;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  return v;
}

// ---- Algorithm 1 (tree-pruning form) run by one lane ----------------------------
// Builds the pruned view of the sorted active set act[0..n) into `view`.
// Returns the view length; *root_used receives the root usage bit (Sec. 9);
// *flops / *n_prim / *n_op describe one evaluation of the view.
struct ViewInfo {
  int n_view, root_used, n_prim, n_op;
  uint32_t flops;
  int err;
};

__device__ __forceinline__ ViewInfo build_view(const DevScene &sc, const uint32_t *act, int n, uint32_t *view,
                               uint32_t *bstk, int stack_cap, uint32_t *vaddr = nullptr) {
  ViewInfo vi = {0, 0, 0, 0, 0u, 0};
  int sp = 0;
  int nv = 0;
  const uint32_t NO = 0x7FFFFFFFu;  // no ancestor: above every address
  auto anc_of = [&](uint32_t b) -> uint32_t { uint32_t a = blob_anc(b); return a == kNoAnc ? NO : a; };
  for (int i = 0; i < n; ++i) {
    const uint32_t P = act[i];
    uint32_t nb = __ldg(sc.blob + P);
    uint32_t anc = anc_of(nb);
    uint32_t u = 1;
    uint32_t isl = blob_isleft(nb);
    {
      const uint32_t code = prim_view_code(blob_kind(nb));
      if (vaddr) vaddr[nv] = P;
      view[nv++] = (code << kViewCodeShift) | kViewGlobal | __ldg(sc.rec_off + P);
      vi.flops += node_flops(code);
      vi.n_prim++;
    }
    if (sp > 0) anc = min(anc, bstk[sp - 1] & 0x7FFFFFFFu);
    const uint32_t next = i + 1 < n ? act[i + 1] : 0u;
    for (int guard = 0;; ++guard) {
      if (i + 1 < n) {
        if (anc > next) break;
      } else if (sp == 0 && anc == NO) {
        break;
      }
      if (anc >= (uint32_t)sc.n_nodes || guard > sc.n_nodes) { vi.err = 1; return vi; }
      const uint32_t pop = anc;
      const uint32_t ab = __ldg(sc.blob + pop);
      const uint32_t a_anc = anc_of(ab);
      const uint32_t m = blob_igm(ab);
      bool popped = false;
      if (sp > 0) {
        const uint32_t c = bstk[sp - 1];
        const uint32_t c_anc = c & 0x7FFFFFFFu;
        if (pop == c_anc || (a_anc >= c_anc && (a_anc == NO || blob_isleft(ab)))) {
          // popRequiredA or popRequiredB: the operator has both operands.
          const uint32_t b = ((c >> 31) << 1) | u;
          --sp;
          const bool ok = ((~b) & m & 3u) == 0u;
          const uint32_t kind = blob_kind(ab);
          uint32_t code;
          if (ok && b == 3u) code = kind - ST_OP_UNION + V_UNION;
          else if (!ok || b == 0u) code = V_INF;
          else code = b == 1u ? V_RIGHT : V_LEFT;
          if (vaddr) vaddr[nv] = pop;
          view[nv++] = (code << kViewCodeShift) | kViewGlobal | __ldg(sc.rec_off + pop);
          vi.flops += node_flops(code);
          vi.n_op++;
          u = (ok && b != 0u) ? 1u : 0u;
          popped = true;
        }
      }
      if (!popped) {
        // Lone operand passing through an operator (Sec. 9 usage rule).
        const uint32_t b = isl ? (u << 1) : u;
        const bool ok = ((~b) & m & 3u) == 0u;
        u = (ok && b != 0u) ? 1u : 0u;
      }
      nb = ab;
      isl = blob_isleft(ab);
      anc = a_anc;
      if (sp > 0) anc = min(anc, bstk[sp - 1] & 0x7FFFFFFFu);
    }
    if (sp >= stack_cap) { vi.err = 2; return vi; }
    bstk[sp++] = anc | (u << 31);
  }
  vi.n_view = nv;
  vi.root_used = sp == 1 ? (int)(bstk[0] >> 31) : 0;
  if (sp != 1) vi.err = 1;
  return vi;
}

// ---- pruned view by lowest common ancestors (warp-collective) -------------------
// The same view as Algorithm 1, built for a GPU warp.  In post-order, the
// operators that Algorithm 1 emits (those with active primitives under both
// operands) are exactly the lowest common ancestors X_i of consecutive active
// primitives A_i < A_i+1, and the view is A and X merged in address order.
// A usage bit climbing from a view node v to its view parent X survives the
// lone-operand nodes in between iff blk(v) >= X, so the usage rewrite of
// Sec. 9 needs no tree walk.  The active set is processed in chunks of
// kViewChunk entries staged in shared memory:
//   phase 1 (all lanes): X_i = first ancestor of A_i at or above A_i+1, by
//     binary lifting (four interleaved searches per lane), and the words the
//     merge needs;
//   phase 2 (lane 0, shared memory only): merge in address order with a
//     value stack (usage, blk, height) and a stack of pending X_i carrying
//     their own words; emit view words, operator codes and the unsorted
//     level schedule;
// then phase 3 (all lanes): counting sort of the operators by height into
// `ops` / `lvl_off` for the tail mode.
// Returns the view info in every lane; *n_lvl_out = levels of the schedule
// (0 when it does not fit kMaxLevels or 16-bit indices).
constexpr int kViewChunk = 128;
struct ViewChunk {       // shared staging of one chunk (warp 0 of a CTA)
  uint4 a[kViewChunk];   // (X_i, blk(X_i), blk(A_i), kind(X_i) | ignoreMod(X_i) << 8)
  uint2 b[kViewChunk];   // (view word of A_i, global flag | record offset of X_i)
};

template <bool kAddr>
__device__ __forceinline__ ViewInfo build_view_lca(const DevScene &sc, const uint32_t *act, int n, uint32_t *view,
                                                   ViewChunk &ch, uint2 *ops, uint2 *sort_tmp, int *lvl_off,
                                                   int *lvl_cur, uint32_t *stk, int stack_cap, uint32_t *vaddr,
                                                   int *n_lvl_out) {
  const int lane = threadIdx.x & 31;
  constexpr uint32_t kNone = 0xFFFFFFFFu;
  constexpr int kPer = kViewChunk / 32;
  ViewInfo vi = {0, 0, 0, 0, 0u, 0};
  int nop = 0, maxh = 0;
  // lane 0's merge state
  // stk: 16-byte aligned, 6 (stack_cap + 2) words
  uint4 *ps = reinterpret_cast<uint4 *>(stk);                       // pending operators: (X, blk, kind | igm << 8, word)
  uint2 *vs = reinterpret_cast<uint2 *>(stk + 4 * (stack_cap + 2)); // value stack: (blk | u << 23 | h << 24, index)
  int vsp = 0, psp = 0, nv = 0;
  uint32_t leaf_flops = 0;   // per lane, reduced after the chunks
  uint2 vt0 = make_uint2(0u, 0u), vt1 = make_uint2(0u, 0u);   // cached value-stack top, second
  uint4 pt = make_uint4(0u, 0u, 0u, 0u);                       // cached pending-operator top
  if (n < 1) vi.err = 1;
  for (int c0 = 0; c0 < n; c0 += kViewChunk) {
    // ---- phase 1 ----
    uint32_t a[kPer], nxt[kPer], x[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = c0 + q * 32 + lane;
      a[q] = i < n ? act[i] : 0u;
      nxt[q] = i + 1 < n ? act[i + 1] : 0u;   // 0: no search
      x[q] = a[q];
    }
    for (int k = sc.lift_levels - 1; k >= 0; --k) {
      const uint32_t *lk = sc.lift + (size_t)k * (uint32_t)sc.n_nodes;
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        if (nxt[q]) {
          const uint32_t y = __ldg(lk + x[q]);
          if (y < nxt[q]) x[q] = y;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = c0 + q * 32 + lane;
      if (i < n) {
        const uint32_t ab = __ldg(sc.blob + a[q]);
        const uint32_t leaf = (prim_view_code(blob_kind(ab)) << kViewCodeShift) | kViewGlobal | __ldg(sc.rec_off + a[q]);
        const uint32_t lb = __ldg(sc.blk + a[q]);
        uint32_t X = kNone, xw = 0u, xblk = kNoAnc, xrec = 0u;
        if (nxt[q]) {
          X = __ldg(sc.lift + x[q]);   // parent of the highest ancestor below A_i+1
          if (X < (uint32_t)sc.n_nodes) {
            const uint32_t xb = __ldg(sc.blob + X);
            xw = blob_kind(xb) | (blob_igm(xb) << 8);
            xblk = __ldg(sc.blk + X);
            xrec = __ldg(sc.rec_off + X);
          }
        }
        ch.a[q * 32 + lane] = make_uint4(X, min(xblk, kNoAnc), min(lb, kNoAnc), xw);
        ch.b[q * 32 + lane] = make_uint2(leaf, kViewGlobal | xrec);
        leaf_flops += node_flops(prim_view_code(blob_kind(ab)));
      }
    }
    __syncwarp();
    // ---- phase 2 ----
    // The top two value-stack entries (vt0 = top) and the top pending
    // operator (pt) live in registers; deeper entries stay in shared memory
    // at their own indices.  This keeps the merge's dependency chain in
    // registers.
    if (lane == 0) {
      const int c1 = min(n, c0 + kViewChunk);
      for (int i = c0; i < c1 && !vi.err; ++i) {
        const uint4 t = ch.a[i - c0];
        const uint2 w = ch.b[i - c0];
        if (vsp >= stack_cap + 2) { vi.err = 2; break; }
        if (kAddr) vaddr[nv] = act[i];
        view[nv] = w.x;
        if (vsp >= 2) vs[vsp - 2] = vt1;
        vt1 = vt0;
        vt0 = make_uint2(t.z | (1u << 23), (uint32_t)nv);
        ++vsp;
        ++nv;
        const uint32_t xnext = i + 1 < n ? t.x : kNone;
        if (i + 1 < n && xnext >= (uint32_t)sc.n_nodes) { vi.err = 1; break; }
        while (psp > 0 && pt.x < xnext) {
          const uint4 pj = pt;
          --psp;
          if (psp > 0) pt = ps[psp - 1];
          if (vsp < 2) { vi.err = 1; break; }
          const uint2 R = vt0, Lv = vt1;
          vsp -= 2;
          const uint2 below = vsp >= 1 ? vs[vsp - 1] : make_uint2(0u, 0u);
          const uint32_t X = pj.x;
          const uint32_t uL = (((Lv.x >> 23) & 1u) && (Lv.x & kNoAnc) >= X) ? 1u : 0u;
          const uint32_t uR = (((R.x >> 23) & 1u) && (R.x & kNoAnc) >= X) ? 1u : 0u;
          const uint32_t b = (uL << 1) | uR, m = (pj.z >> 8) & 3u, kind = pj.z & 31u;
          const bool ok = ((~b) & m & 3u) == 0u;
          const bool keep = ok && b == 3u;
          const uint32_t code = keep ? kind - ST_OP_UNION + V_UNION
                                     : ((!ok || b == 0u) ? (uint32_t)V_INF : (b == 1u ? (uint32_t)V_RIGHT : (uint32_t)V_LEFT));
          if (kAddr) vaddr[nv] = X;
          view[nv] = (code << kViewCodeShift) | pj.w;
          vi.flops += keep ? (kind <= ST_OP_DIFF ? kFlopsCompactOp : kFlopsSharpOp) : 0u;
          const uint32_t h = min(max(Lv.x >> 24, R.x >> 24) + 1u, 255u);
          maxh = max(maxh, (int)h);
          ops[nop++] = make_uint2((uint32_t)nv | (Lv.y << 16), (R.y & 0xFFFFu) | (h << 16));
          const uint32_t u = (ok && b != 0u) ? 1u : 0u;
          vt1 = below;
          vt0 = make_uint2(pj.y | (u << 23) | (h << 24), (uint32_t)nv);
          ++vsp;
          ++nv;
        }
        if (vi.err) break;
        if (i + 1 < n) {
          if (psp >= stack_cap + 2) { vi.err = 2; break; }
          if (psp >= 1) ps[psp - 1] = pt;
          pt = make_uint4(t.x, t.y, t.w, w.y);
          ++psp;
        }
      }
    }
    __syncwarp();
    if (__shfl_sync(0xFFFFFFFFu, vi.err, 0)) break;
  }
  if (lane == 0) {
    if (!vi.err) {
      if (vsp != 1 || psp != 0) vi.err = 1;
      else vi.root_used = (((vt0.x >> 23) & 1u) && (vt0.x & kNoAnc) == kNoAnc) ? 1 : 0;
    }
    vi.n_view = nv;
    vi.n_prim = n;
    vi.n_op = nop;
  }
  vi.n_view = __shfl_sync(0xFFFFFFFFu, vi.n_view, 0);
  vi.root_used = __shfl_sync(0xFFFFFFFFu, vi.root_used, 0);
  vi.n_prim = __shfl_sync(0xFFFFFFFFu, vi.n_prim, 0);
  vi.n_op = __shfl_sync(0xFFFFFFFFu, vi.n_op, 0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) leaf_flops += __shfl_xor_sync(0xFFFFFFFFu, leaf_flops, o);
  vi.flops = __shfl_sync(0xFFFFFFFFu, vi.flops, 0) + leaf_flops;
  vi.err = __shfl_sync(0xFFFFFFFFu, vi.err, 0);
  nop = __shfl_sync(0xFFFFFFFFu, nop, 0);
  maxh = __shfl_sync(0xFFFFFFFFu, maxh, 0);
  int n_lvl = 0;
  if (!vi.err && vi.root_used && vi.n_view <= 65535 && maxh <= kMaxLevels) {
    for (int h = lane; h <= kMaxLevels; h += 32) lvl_off[h] = 0;
    __syncwarp();
    for (int k = lane; k < nop; k += 32) atomicAdd(&lvl_off[ops[k].y >> 16], 1);
    __syncwarp();
    if (lane == 0) {
      int acc = 0;
      lvl_off[0] = 0;
      for (int h = 1; h <= maxh; ++h) {
        const int c = lvl_off[h];
        lvl_cur[h] = acc;
        acc += c;
        lvl_off[h] = acc;
      }
    }
    __syncwarp();
    for (int k = lane; k < nop; k += 32) {
      const uint2 o = ops[k];
      const int pos = atomicAdd(&lvl_cur[o.y >> 16], 1);
      sort_tmp[pos] = make_uint2(o.x, o.y & 0xFFFFu);
    }
    __syncwarp();
    for (int k = lane; k < nop; k += 32) ops[k] = sort_tmp[k];
    __syncwarp();
    n_lvl = maxh;
  }
  *n_lvl_out = n_lvl;
  return vi;
}

// Parameter cache fill (Sec. 8 "local pruned tree view"): the records of the
// view's nodes are copied into the view's shared cache, warp-cooperatively,
// in view order until the cache is full; the remaining nodes keep reading
// the scene's global records.  Record words needed per node code.
__device__ __forceinline__ int code_words(uint32_t code) {
  // record words of codes 0..15 as 4-bit fields (1 4 3 1 1 1 0 0 0 0 0 0 2 4 5 7),
  // code 16 (bounded quadric) 5: no indexed jump per staged node
  // (a CTA-split LOAD stages the 32 lanes' float2 values: 16 words)
  constexpr unsigned long long kWords = 0x7542000000111341ull;
  return code < 16 ? (int)((kWords >> (4 * code)) & 15u) : (code == V_QUADRIC ? 5 : (code == V_LOAD ? 16 : 0));
}

// ---- staged evaluation of views held in global memory ------------------------------
// When a launch's views do not fit in shared memory, reading a view word and
// then its node's record from L2 costs two dependent memory latencies per
// node, which the interpreter's one-node-ahead load of the next word cannot
// hide.  The staged form has the warp fetch the next chunk of up to 32 nodes
// at once: one coalesced load of their view words (one per lane), then
// asynchronous copies (cp.async, 16 bytes each, all lanes at once) of the
// record words of the nodes whose records are not in the shared parameter
// cache, into the warp's shared stage buffer; the chunk is then evaluated from
// shared memory.  One round of latency per chunk instead of one per node.

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int R, class T, class Stk, int kFam>
__device__ __forceinline__ void eval_view_staged(const uint32_t *view, int n_view, const RecSrc &src,
                                                 const T (&p)[R][3], T (&acc)[R], Stk &stk, float4 *stage) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = T(0.f);
  int sp = 0;
  // staged records are read through the "global" side of the record source
  const RecSrc ss{stage, src.dc};
  for (int i0 = 0; i0 < n_view;) {
    const int i = i0 + lane;
    uint32_t w = i < n_view ? view[i] : 0u;
    const int nw = (w & kViewGlobal) ? code_words(w >> kViewCodeShift) : 0;
    int x = nw;   // inclusive prefix sum of the words to stage
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    const bool fits = x <= kStageWords;   // a prefix of the lanes (x never decreases)
    const int nb = min(n_view - i0, __popc(__ballot_sync(0xFFFFFFFFu, fits)));
    if (fits && nw > 0) {
      const int off = x - nw;
      const float4 *g = src.rec + (w & kViewOffMask);
      for (int k = 0; k < nw; ++k) cp_async16(stage + off + k, g + k);
      w = (w & ~kViewOffMask) | (uint32_t)off;
    }
    cp_async_wait_all();
    __syncwarp();
    for (int j = 0; j < nb; ++j) {
      const uint32_t wj = __shfl_sync(0xFFFFFFFFu, w, j);
      eval_node<R, T, Stk, kFam>(wj >> kViewCodeShift, rec_ptr(ss, wj), p, acc, stk, sp);
    }
    __syncwarp();   // the next chunk overwrites the stage
    i0 += nb;
  }
}

__device__ __forceinline__ void fill_dcache(uint32_t *view, int n_view, const float4 *rec, float4 *dc, int cap) {
  const int lane = threadIdx.x & 31;
  int base = 0;
  for (int b = 0; b < n_view; b += 32) {
    const int i = b + lane;
    const uint32_t w = i < n_view ? view[i] : 0u;
    const int nw = i < n_view ? code_words(w >> kViewCodeShift) : 0;
    int x = nw;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    const int off = base + x - nw;
    if (nw > 0 && off + nw <= cap) {
      const float4 *sp = rec + (w & kViewOffMask);
      for (int k = 0; k < nw; ++k) dc[off + k] = __ldg(sp + k);
      view[i] = (w & ~(kViewGlobal | kViewOffMask)) | (uint32_t)off;
    }
    base += __shfl_sync(0xFFFFFFFFu, x, 31);
    if (base >= cap) break;
  }
  __syncwarp();
}

// ---- subfrustum preparation (warp 0) -------------------------------------------
struct SegState {   // registers of warp 0, kept across the subfrustums of a tile
  uint32_t next;
  int n_act, cur;
  float z_end, maxze;
};

struct SubInfo {    // one prepared subfrustum, published in shared memory
  float z_begin, z_end;
  int n_view, root_used, n_prim, n_op, err, done;
  int n_lvl;          // operator levels of the schedule (0: tail mode unavailable)
  uint32_t flops;      // n_prim, n_op, flops: the subfrustum's pruned view (Algorithm 1,
                       // Sec. 9 usage); n_view and flops_eval: the view evaluated, without
                       // the subtrees whose values that view discards
  uint32_t flops_eval;
};

// Level schedule of a view for the warp-wide evaluation of a single point:
// operators grouped by their height in the pruned tree, each with the view
// indices of its operands.  One lane; uses the Algorithm 1 stack memory.
// Returns the number of levels, or 0 when there are more than kMaxLevels or
// the view does not fit 16-bit indices.
__device__ __forceinline__ int build_schedule(const uint32_t *view, int n_view, uint2 *ops, int *lvl_off, uint32_t *bstk,
                              int stack_cap) {
  if (n_view <= 0 || n_view > 65535) return 0;
  // lvl_off doubles as the per-level counter array during the build.
  for (int h = 0; h <= kMaxLevels; ++h) lvl_off[h] = 0;
  int sp = 0, max_lvl = 0;
  // pass 1: heights and level counts (stack entry: index | level << 16)
  for (int i = 0; i < n_view; ++i) {
    const uint32_t code = view[i] >> kViewCodeShift;
    if (is_prim_code(code)) {
      if (sp >= stack_cap) return 0;
      bstk[sp++] = (uint32_t)i;
    } else {
      const uint32_t r = bstk[--sp], l = bstk[--sp];
      const int lev = (int)max(l >> 16, r >> 16) + 1;
      if (lev > kMaxLevels) return 0;
      lvl_off[lev]++;
      max_lvl = max(max_lvl, lev);
      bstk[sp++] = (uint32_t)i | ((uint32_t)lev << 16);
    }
  }
  // exclusive offsets: lvl_off[h] = start of level h+1 (levels are 1-based)
  int acc = 0;
  for (int h = 1; h <= max_lvl; ++h) {
    const int c = lvl_off[h];
    lvl_off[h - 1] = acc;
    acc += c;
  }
  lvl_off[max_lvl] = acc;
  // pass 2: place operators (cursor per level kept in lvl_off, restored after)
  sp = 0;
  for (int i = 0; i < n_view; ++i) {
    const uint32_t code = view[i] >> kViewCodeShift;
    if (is_prim_code(code)) {
      bstk[sp++] = (uint32_t)i;
    } else {
      const uint32_t r = bstk[--sp], l = bstk[--sp];
      const int lev = (int)max(l >> 16, r >> 16) + 1;
      ops[lvl_off[lev - 1]++] = make_uint2((uint32_t)i | ((l & 0xFFFFu) << 16), r & 0xFFFFu);
      bstk[sp++] = (uint32_t)i | ((uint32_t)lev << 16);
    }
  }
  // the cursors now hold the level ends; shift back to level starts
  for (int h = max_lvl; h >= 1; --h) lvl_off[h] = lvl_off[h - 1];
  lvl_off[0] = 0;
  return max_lvl;
}


// ---- CTA-split evaluation of a large view -------------------------------------------
// Algorithm 3 over a view in post-order, cut into kWarps contiguous segments
// (node count split evenly): warp w evaluates segment w for the owner warp's
// points while the other warps evaluate theirs, and the owner then combines
// the pieces.  A node whose subtree crosses a segment boundary (a proper
// ancestor of the node just before a boundary) is a top node; the other
// children of top nodes are forest roots, each the root of a complete subtree
// inside one segment.  Segment w's stream is its nodes in order with the top
// nodes replaced by a STORE for each of their children that is a forest root
// of the same segment (right child first: it is the running value, the left
// one lies just below it), followed by a STORE for every forest root still on
// the stack at the segment's end (topmost first): its stack never holds more
// than the full evaluation's, and the values leave it in a known order.  The
// top program is the top nodes and forest roots in view order, the roots as
// LOADs of their output slots: the post-order of the tree above the segments.
// Every node computes the same operations on the same operands as in the full
// evaluation, so the value is bit for bit the same.
struct CtaInfo {   // CTA split of one view buffer (shared memory)
  int n_top;       // top program words (0: no split for this view)
  int off[kWarps], len[kWarps], slot[kWarps];   // segment streams and their first output slots
  int stt[kWarps], ntr[kWarps];   // build: STOREs at top nodes, trailing STOREs per segment
};
struct CtaSync {   // CTA-split protocol of one subfrustum (shared memory)
  int flag;        // 0 none, 1 requested (owner waits for the helpers), 2 running, 3 abandoned
  int join;        // helpers that handed their rays over
  int cmd;         // owner -> helpers at each pass: 1 evaluate, kCtaDone finished
  int w0in;        // warp 0 (the view builder) is marching this subfrustum
  int own, nh;     // at the end: the owner warp and its hit count
  int vb;          // the subfrustum's view buffer
};
// CTA-split state of a CTA, at namespace scope so that march_sub reaches it
// without carrying pointers through the lockstep loop (registers).
struct CtaShared {
  CtaInfo info[2];   // per view buffer
  CtaSync sync[3];   // per subfrustum slot
  const uint32_t *cseg[2], *ctop[2];
  float4 *crec;
};
__shared__ CtaShared s_ctash;

// Warp-collective (warp 0, after the parameter cache fill, so that segment
// words are the view's own); node scratch and outputs in the work area.
__device__ __forceinline__ void build_cta_split(const uint32_t *view, int n, const uint2 *ops, int nop, const float4 *rec,
                                             const float4 *dc, int vb, const CtaWork &C, int view_cap, CtaInfo *out) {
  constexpr uint32_t kNone = 0xFFFFFFFFu, kTop = 1u, kRoot = 2u, kTrail = 0x80000000u;
  const int lane = threadIdx.x & 31;
  uint32_t *par = C.cscr, *lft = C.cscr + view_cap, *flg = C.cscr + 2 * (size_t)view_cap,
           *slt = C.cscr + 3 * (size_t)view_cap;
  uint32_t *seg = pick(C.cseg, vb), *top = pick(C.ctop, vb);
  const int seg_cap = view_cap + kCtaOutMax;
  // (no local arrays: the per-segment values go to *out in shared memory)
  auto bnd = [n](int w) { return (int)(((long long)n * w) / kWarps); };
  if (lane == 0) out->n_top = 0;
  // parents and left children from the operators' operand indices (the right
  // child of an operator at i is i - 1)
  for (int i = lane; i < n; i += 32) { par[i] = kNone; flg[i] = 0u; }
  __syncwarp();
  for (int k = lane; k < nop; k += 32) {
    const uint2 o = ops[k];
    const uint32_t t = o.x & 0xFFFFu, l = o.x >> 16, r = o.y & 0xFFFFu;
    if (t < (uint32_t)n && l < t && r < t) {
      par[l] = t;
      par[r] = t;
      lft[t] = l;
    }
  }
  __syncwarp();
  if (lane >= 1 && lane < kWarps) {   // top nodes: ancestors of the node before each boundary
    uint32_t t = par[bnd(lane) - 1];
    for (int it = 0; t != kNone && it < n; ++it) {
      flg[t] = kTop;
      t = par[t];
    }
  }
  __syncwarp();
  for (int i = lane; i < n; i += 32) {
    const uint32_t p = par[i];
    if (!(flg[i] & kTop) && p != kNone && (flg[p] & kTop)) flg[i] = kRoot;
  }
  __syncwarp();
  int off = 0, slot = 0;
  bool ok = true;
#pragma unroll 1
  for (int w = 0; w < kWarps; ++w) {
    const int lo = bnd(w), hi = bnd(w + 1);
    int pos = 0, sst = 0, ntr = 0;
    for (int c0 = lo; c0 < hi; c0 += 32) {
      const int i = c0 + lane;
      const bool v = i < hi;
      const uint32_t f = v ? flg[i] : 0u;
      int nw = 0, ns = 0;
      bool sr = false, sl = false, trailing = false;
      uint32_t l = 0u;
      if (v) {
        if (f & kTop) {
          l = lft[i];
          sr = i - 1 >= lo && (flg[i - 1] & kRoot);
          sl = (int)l >= lo && (flg[l] & kRoot);
          ns = nw = (int)sr + (int)sl;
        } else {
          nw = 1;
          trailing = (f & kRoot) && par[i] >= (uint32_t)hi;
        }
      }
      int xw = nw, xs = ns;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int yw = __shfl_up_sync(0xFFFFFFFFu, xw, o), ys = __shfl_up_sync(0xFFFFFFFFu, xs, o);
        if (lane >= o) { xw += yw; xs += ys; }
      }
      const int pw = off + pos + xw - nw, ps = slot + sst + xs - ns;
      if (v && pw + nw <= seg_cap) {
        if (f & kTop) {
          if (sr) { seg[pw] = (uint32_t)V_STORE << kViewCodeShift; slt[i - 1] = (uint32_t)ps; }
          if (sl) { seg[pw + (int)sr] = (uint32_t)V_STORE << kViewCodeShift; slt[l] = (uint32_t)(ps + (int)sr); }
        } else {
          seg[pw] = view[i];
        }
      }
      const uint32_t tm = __ballot_sync(0xFFFFFFFFu, trailing);
      if (trailing) slt[i] = kTrail | (uint32_t)(ntr + __popc(tm & lanemask_lt()));
      ntr += __popc(tm);
      pos += __shfl_sync(0xFFFFFFFFu, xw, 31);
      sst += __shfl_sync(0xFFFFFFFFu, xs, 31);
    }
    for (int j = lane; j < ntr; j += 32)
      if (off + pos + j < seg_cap) seg[off + pos + j] = (uint32_t)V_STORE << kViewCodeShift;
    pos += ntr;
    if (lane == 0) {
      out->off[w] = off;
      out->len[w] = pos;
      out->slot[w] = slot;
      out->stt[w] = sst;
      out->ntr[w] = ntr;
    }
    off += pos;
    slot += sst + ntr;
  }
  if (off > seg_cap || slot > kCtaOutMax) ok = false;
  __syncwarp();
  // top program: top nodes (operators, records copied next to the program)
  // and forest roots (LOADs of their slots) in view order
  int ntop = 0;
  for (int c0 = 0; c0 < n && ok; c0 += 32) {
    const int i = c0 + lane;
    const uint32_t f = i < n ? flg[i] : 0u;
    const uint32_t mm = __ballot_sync(0xFFFFFFFFu, f != 0u);
    const int p = ntop + __popc(mm & lanemask_lt());
    if (f != 0u && p < kCtaTopMax) {
      uint32_t word;
      if (f & kTop) {
        const uint32_t vw = view[i], code = vw >> kViewCodeShift;
        if (code_words(code) > 0) {   // a compact operator: one record word
          const int ri = vb * kCtaTopMax + p;
          C.crec[ri] = *rec_ptr(RecSrc{rec, dc}, vw);
          word = (code << kViewCodeShift) | kViewGlobal | (uint32_t)ri;
        } else {
          word = code << kViewCodeShift;
        }
      } else {
        const int w = (i >= bnd(1)) + (i >= bnd(2)) + (i >= bnd(3));
        uint32_t sl = slt[i];
        if (sl & kTrail) sl = (uint32_t)(out->slot[w] + out->stt[w] + out->ntr[w] - 1 - (int)(sl & ~kTrail));
        word = ((uint32_t)V_LOAD << kViewCodeShift) | kViewGlobal | (uint32_t)(2 * kCtaTopMax + 16 * (int)sl);
      }
      top[p] = word;
    }
    ntop += __popc(mm);
  }
  if (ntop > kCtaTopMax) ok = false;
  __syncwarp();
  if (lane == 0) out->n_top = ok ? ntop : 0;
  __syncwarp();
}

// ---- subtrees whose values the pruned view discards ------------------------------
// The usage rewrite of Sec. 9 turns an operator with an unusable operand into
// "right operand", "left operand" or "+inf": the discarded operand's whole
// subtree is evaluated for nothing (with intersections and differences among
// the operators, 50-70 % of a subfrustum's view on the synthetic scenes).
// Liveness from the root down, by levels of the view's schedule (operators
// sorted by height, built with the view): from the top level down, each
// operator passes its liveness to the operands it uses, all operators of a
// level at once.  The view of the live primitives holds exactly the live
// nodes that are primitives or keep their operator (every operator whose
// operands are both live keeps them; the rewritten operators vanish with
// their discarded operands), in the same post-order, so every value computed
// is the same bit for bit.  That view is made here by compacting the first
// one instead of building it again: kept nodes move to their rank among the
// kept nodes; a live "left" / "right" operator hands its parent the node of
// the operand it passes on; heights and the level schedule are recomputed
// bottom-up over the old levels (operands sit on lower levels).
// Warp-collective.  scratch: 4 n + 2 bytes (live flags, the node that carries
// each value, new heights), dead once the schedule is sorted into it.
// Returns the new view size, 0 when nothing is discarded (the view is left
// as it is).
__device__ __forceinline__ int compact_live_view(uint32_t *view, int n, uint2 *ops, int *lvl_off, int *lvl_cur,
                                                 int n_lvl, uint2 *scratch, int *nop_out, int *nlvl_out,
                                                 uint32_t *flops_out, uint32_t *vaddr) {
  const int lane = threadIdx.x & 31;
  uint8_t *live = reinterpret_cast<uint8_t *>(scratch);
  uint16_t *rep = reinterpret_cast<uint16_t *>(live + ((n + 1) & ~1));
  uint8_t *hn = reinterpret_cast<uint8_t *>(rep + n);
  if (lane == 0) live[n - 1] = 1;   // the root (post-order: last)
  __syncwarp();
  for (int h = n_lvl; h >= 1; --h) {
    for (int k = lvl_off[h - 1] + lane; k < lvl_off[h]; k += 32) {
      const uint2 o = ops[k];
      const uint32_t t = o.x & 0xFFFFu, l = o.x >> 16, r = o.y & 0xFFFFu;
      const uint32_t code = view[t] >> kViewCodeShift;
      const bool keep = code <= V_SDIFF, on = live[t] != 0;
      live[l] = (uint8_t)(on && (keep || code == V_LEFT));
      live[r] = (uint8_t)(on && (keep || code == V_RIGHT));
    }
    __syncwarp();
  }
  // new positions; primitives carry their own values at height 0
  int nk = 0;
  uint32_t fl = 0;
  for (int c = 0; c < n; c += 32) {
    const int i = c + lane;
    const uint32_t code = i < n ? view[i] >> kViewCodeShift : (uint32_t)V_INF;
    const bool prim = i < n && is_prim_code(code);
    const bool kept = i < n && live[i] != 0 && (prim || code <= V_SDIFF);
    const uint32_t km = __ballot_sync(0xFFFFFFFFu, kept);
    if (kept) {
      rep[i] = (uint16_t)(nk + __popc(km & lanemask_lt()));
      if (prim) hn[i] = 0;
      fl += node_flops(code);
    }
    nk += __popc(km);
  }
  __syncwarp();
  if (nk >= n) return 0;
  // operands and heights of the kept operators, level by level; the new
  // entries are written over the old ones (never ahead of the reads)
  int nop = 0, maxh = 0;
  for (int h = 1; h <= n_lvl; ++h) {
    const int e = lvl_off[h];
    for (int k0 = lvl_off[h - 1]; k0 < e; k0 += 32) {
      const int k = k0 + lane;
      uint2 o = make_uint2(0u, 0u);
      bool kept = false;
      if (k < e) {
        o = ops[k];
        const uint32_t t = o.x & 0xFFFFu, l = o.x >> 16, r = o.y & 0xFFFFu;
        if (live[t]) {
          const uint32_t code = view[t] >> kViewCodeShift;
          if (code <= V_SDIFF) {
            const uint32_t h2 = max(hn[l], hn[r]) + 1u;
            hn[t] = (uint8_t)h2;
            maxh = max(maxh, (int)h2);
            o = make_uint2((uint32_t)rep[t] | ((uint32_t)rep[l] << 16), (uint32_t)rep[r] | (h2 << 16));
            kept = true;
          } else if (code == V_LEFT) {
            rep[t] = rep[l];
            hn[t] = hn[l];
          } else if (code == V_RIGHT) {
            rep[t] = rep[r];
            hn[t] = hn[r];
          }
        }
      }
      const uint32_t km = __ballot_sync(0xFFFFFFFFu, kept);
      __syncwarp();
      if (kept) ops[nop + __popc(km & lanemask_lt())] = o;
      nop += __popc(km);
    }
    __syncwarp();
  }
  // the view itself, in place
  int out = 0;
  for (int c = 0; c < n; c += 32) {
    const int i = c + lane;
    const uint32_t v = i < n ? view[i] : 0u;
    const uint32_t va = (vaddr && i < n) ? vaddr[i] : 0u;
    const uint32_t code = v >> kViewCodeShift;
    const bool kept = i < n && live[i] != 0 && (is_prim_code(code) || code <= V_SDIFF);
    const uint32_t km = __ballot_sync(0xFFFFFFFFu, kept);
    __syncwarp();
    if (kept) {
      const int pos = out + __popc(km & lanemask_lt());
      view[pos] = v;
      if (vaddr) vaddr[pos] = va;
    }
    out += __popc(km);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fl += __shfl_xor_sync(0xFFFFFFFFu, fl, o);
    maxh = max(maxh, __shfl_xor_sync(0xFFFFFFFFu, maxh, o));
  }
  __syncwarp();
  // level schedule (counting sort by the new heights; scratch is free now)
  for (int h = lane; h <= kMaxLevels; h += 32) lvl_off[h] = 0;
  __syncwarp();
  for (int k = lane; k < nop; k += 32) atomicAdd(&lvl_off[ops[k].y >> 16], 1);
  __syncwarp();
  if (lane == 0) {
    int acc = 0;
    lvl_off[0] = 0;
    for (int h = 1; h <= maxh; ++h) {
      const int c = lvl_off[h];
      lvl_cur[h] = acc;
      acc += c;
      lvl_off[h] = acc;
    }
  }
  __syncwarp();
  for (int k = lane; k < nop; k += 32) {
    const uint2 o = ops[k];
    const int pos = atomicAdd(&lvl_cur[o.y >> 16], 1);
    scratch[pos] = make_uint2(o.x, o.y & 0xFFFFu);
  }
  __syncwarp();
  for (int k = lane; k < nop; k += 32) ops[k] = scratch[k];
  __syncwarp();
  *nop_out = nop;
  *nlvl_out = maxh;
  *flops_out = fl;
  return nk;
}

// Tracking active primitives (Sec. 8): discard those with z_e <= z_end,
// fetch new ones from the depth-sorted list while the four conditions hold,
// keep the set sorted by node address; then Algorithm 1 (one lane) builds the
// pruned view into `view` (not when !build: replaying a tile's segmentation).
// Warp-collective; lane 0 writes *out.
__device__ __forceinline__ void prepare_sub(SegState &sg, const CtaWork &C, const DevScene &sc, const TraceParams &tp,
                            const float *zin_l, const float *zout_l, const uint32_t *prim_l, uint32_t len,
                            int vb, int stack_slots, int dc_words, SubInfo *out, int *lvl_cur, ViewChunk *vch,
                            unsigned long long *dbg, bool build, int cta_min, int view_cap, CtaInfo *cta_out,
                            bool prune) {
  uint32_t *view = pick(C.view, vb);
  const int lane = threadIdx.x & 31;
  long long tc = dbg ? clock64() : 0;
  auto lap = [&](int slot) {   // per-phase cycle counters (tile diagnostics)
    if (dbg) {
      const long long t = clock64();
      if (lane == 0) dbg[slot] += (unsigned long long)(t - tc);
      tc = t;
    }
  };
  // ---- discard ----
  {
    int kept = 0;
    float mz = -INFINITY;
    for (int b = 0; b < sg.n_act; b += 32) {
      const int i = b + lane;
      const bool v = i < sg.n_act;
      const float ze = v ? pick(C.act_ze, sg.cur)[i] : -INFINITY;
      const uint32_t ad = v ? pick(C.act, sg.cur)[i] : 0u;
      const bool keep = v && ze > sg.z_end;
      const uint32_t km = __ballot_sync(0xFFFFFFFFu, keep);
      if (keep) {
        const int dst = kept + __popc(km & lanemask_lt());
        pick(C.act, sg.cur ^ 1)[dst] = ad;
        pick(C.act_ze, sg.cur ^ 1)[dst] = ze;
        mz = fmaxf(mz, ze);
      }
      kept += __popc(km);
    }
    sg.n_act = kept;
    sg.cur ^= 1;
    sg.maxze = warp_max(mz);
    __syncwarp();
  }
  lap(0);
  SubInfo info;
  info.done = (sg.n_act == 0 && sg.next >= len) ? 1 : 0;
  info.err = 0;
  info.n_view = info.root_used = info.n_prim = info.n_op = info.n_lvl = 0;
  info.flops = info.flops_eval = 0u;
  info.z_begin = info.z_end = sg.z_end;
  if (!info.done) {
    // ---- fetch (no empty space, depth slab d, max new per turn; no overlap cap) ----
    // Candidates are examined 32 at a time (one per lane) until a condition
    // fails or max_new have been taken.  A tile takes at least an eighth of
    // its list per turn: long lists (clustered primitives) otherwise split
    // into many subfrustums, each marching over a large view (measured on
    // B300: 10k clustered primitives 2.1x faster at 1920x1080, 2.8x at
    // 3840x2160; no change on short lists).
    float z_begin = sg.z_end;
    if (sg.next < len) z_begin = fmaxf(sg.z_end, __ldg(zin_l + sg.next));
    const int max_new = max(tp.max_new, (int)(len >> 3));
    for (int fetched = 0; sg.next < len && fetched < max_new;) {
      const int quota = min(32, max_new - fetched);
      const uint32_t c = sg.next + (uint32_t)lane;
      const bool valid = lane < quota && c < len;
      const float zb = valid ? __ldg(zin_l + c) : INFINITY;
      const float ze = valid ? __ldg(zout_l + c) : -INFINITY;
      const uint32_t pa = valid ? __ldg(prim_l + c) : 0xFFFFFFFFu;
      float run = ze;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(0xFFFFFFFFu, run, o);
        if (lane >= o) run = fmaxf(run, y);
      }
      float excl = __shfl_up_sync(0xFFFFFFFFu, run, 1);
      excl = lane == 0 ? sg.maxze : fmaxf(excl, sg.maxze);
      const bool ok = valid && ((lane == 0 && sg.n_act == 0) ||
                                (zb <= excl && zb - z_begin < tp.depth_slab));
      const uint32_t fail = __ballot_sync(0xFFFFFFFFu, !ok);
      const int take = fail ? __ffs(fail) - 1 : 32;
      const bool taken = lane < take;
      sg.maxze = warp_max(taken ? fmaxf(ze, sg.maxze) : sg.maxze);
      // sorted merge by node address: the taken candidates are sorted
      // across the lanes (bitonic network), then one pass over the active
      // set places every old entry after the new ones below it and counts,
      // for every new entry, the old ones below it (binary searches over
      // sorted lanes, five shuffles each).
      uint32_t key = taken ? pa : 0xFFFFFFFFu;
      float kze = ze;
#pragma unroll
      for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
          const uint32_t ok = __shfl_xor_sync(0xFFFFFFFFu, key, jj);
          const float oz = __shfl_xor_sync(0xFFFFFFFFu, kze, jj);
          const bool keep_min = ((lane & jj) == 0) == ((lane & kk) == 0);
          if (keep_min ? ok < key : ok > key) {
            key = ok;
            kze = oz;
          }
        }
      }
      const uint32_t *A = pick(C.act, sg.cur);
      const float *AZ = pick(C.act_ze, sg.cur);
      uint32_t *B = pick(C.act, sg.cur ^ 1);
      float *BZ = pick(C.act_ze, sg.cur ^ 1);
      int below_new = 0;   // old entries below this lane's new key
      for (int b = 0; b < sg.n_act; b += 32) {
        const int i = b + lane;
        const uint32_t ad = i < sg.n_act ? A[i] : 0xFFFFFFFFu;
        const int m = min(32, sg.n_act - b);
        const int before = lanes_below(key, take, ad);
        below_new += lanes_below(ad, m, key);
        if (i < sg.n_act) {
          B[i + before] = ad;
          BZ[i + before] = AZ[i];
        }
      }
      if (lane < take) {
        B[lane + below_new] = key;
        BZ[lane + below_new] = kze;
      }
      sg.n_act += take;
      sg.cur ^= 1;
      sg.next += (uint32_t)take;
      fetched += take;
      __syncwarp();
      if (take < quota) break;
    }
    sg.z_end = sg.next < len ? fminf(__ldg(zin_l + sg.next), sg.maxze) : sg.maxze;
    info.z_begin = z_begin;
    info.z_end = sg.z_end;
    __syncwarp();
    lap(1);
  }
  if (!info.done && build) {
    // ---- pruned view (the lowest-common-ancestor form of Algorithm 1) ----
    int n_lvl = 0;
    ViewInfo vi = build_view_lca<false>(sc, pick(C.act, sg.cur), sg.n_act, view, *vch, pick(C.ops, vb), C.sort_tmp,
                                        pick(C.lvl_off, vb), lvl_cur, C.bstk, stack_slots, nullptr, &n_lvl);
    info.root_used = vi.root_used;
    info.n_prim = vi.n_prim;
    info.n_op = vi.n_op;
    info.flops = vi.flops;
    if (prune && !vi.err && vi.root_used && n_lvl > 0) {
      // without the subtrees its usage rewrite discards (the view of the live primitives)
      int nop2 = 0, nlvl2 = 0;
      uint32_t fl2 = 0;
      const int n2 = compact_live_view(view, vi.n_view, pick(C.ops, vb), pick(C.lvl_off, vb), lvl_cur, n_lvl,
                                       C.sort_tmp, &nop2, &nlvl2, &fl2, nullptr);
      if (n2 > 0) {
        vi.n_view = n2;
        vi.n_op = nop2;
        vi.flops = fl2;
        n_lvl = nlvl2;
      }
    }
    info.n_view = vi.n_view;
    info.flops_eval = vi.flops;
    info.err = vi.err;
    info.n_lvl = (!vi.err && vi.root_used) ? n_lvl : 0;
    lap(2);
    if (!vi.err && vi.root_used) fill_dcache(view, vi.n_view, sc.rec, pick(C.dc, vb), dc_words);
    lap(3);
    if (cta_min > 0) {
      if (!vi.err && vi.root_used && vi.n_view >= cta_min && vi.n_view <= 65535)
        build_cta_split(view, vi.n_view, pick(C.ops, vb), vi.n_op, sc.rec, pick(C.dc, vb), vb, C, view_cap,
                        cta_out + vb);
      else if (lane == 0)
        cta_out[vb].n_top = 0;
      __syncwarp();
    }
  }
  if (lane == 0) *out = info;
  __syncwarp();
}

// ---- warp-wide evaluation of one point (tail mode) ------------------------------------
// All lanes hold the same point p.  Primitives are evaluated in parallel,
// then operators level by level (operands always sit on lower levels).
// `vals` is per-warp shared memory of at least n_view floats.
template <int kFam>
__device__ __forceinline__ float tail_eval(const uint32_t *view, int n_view, const uint2 *ops, const int *lvl_off, int n_lvl,
                           const RecSrc &src, const float p[3], float *vals) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < n_view; i += 32) {
    const uint32_t w = view[i];
    const uint32_t code = w >> kViewCodeShift;
    if (!is_prim_code(code)) continue;
    const float4 *q = rec_ptr(src, w);
    float v;
    if (code == V_SPHERE) v = sd_sphere<float>(ldrec(q), p);
    else if (code == V_RBOX) v = sd_rbox<float>(ldrec(q), ldrec(q + 1), ldrec(q + 2), ldrec(q + 3), p);
    else if (code == V_CAPSULE) v = sd_capsule<float>(ldrec(q), ldrec(q + 2), p);
    else v = kFam ? sd_further<float, kFam == 2>(code, q, p[0], p[1], p[2]) : INFINITY;
    vals[i] = v;
  }
  __syncwarp();
  for (int h = 0; h < n_lvl; ++h) {
    const int e = lvl_off[h + 1];
    for (int j = lvl_off[h] + lane; j < e; j += 32) {
      const uint2 o = ops[j];
      const int self = (int)(o.x & 0xFFFFu), li = (int)(o.x >> 16), ri = (int)o.y;
      const uint32_t w = view[self];
      const float f0 = vals[li], f1 = vals[ri];
      const float4 *q = rec_ptr(src, w);
      float v;
      const uint32_t code = w >> kViewCodeShift;
      if (code <= V_DIFF) v = op_compact_any<float>(code, ldrec(q), f0, f1);
      else if (code <= V_SDIFF) v = op_sharp_any<float>(code, f0, f1);
      else if (code == V_INF) v = INFINITY;
      else if (code == V_RIGHT) v = f1;
      else v = f0;
      vals[self] = v;
    }
    __syncwarp();
  }
  const float r = vals[n_view - 1];
  __syncwarp();
  return r;
}

// ---- marching one subfrustum: lockstep evaluation with ray refill -----------------
struct MarchCtx {
  const DevCamera *cam;
  const TraceParams *tp;
  const DevOut *out;
  int x0, y0, tw;
};

__device__ __forceinline__ void load_ray(const MarchCtx &M, const CtaWork &C, int r, float z_begin, float &z,
                                         uint32_t &steps, float d[3], float &inv_ld) {
  z = fmaxf(C.ray_z[r], z_begin);
  steps = C.ray_st[r] & 0xFFFFFFu;
  pixel_ray(*M.cam, M.x0 + r % M.tw, M.y0 + r / M.tw, d);
  inv_ld = 1.0f / mul_(M.tp->lipschitz, sqrtf(fma_(d[0], d[0], fma_(d[1], d[1], mul_(d[2], d[2])))));
}

__device__ __forceinline__ void write_miss(const MarchCtx &M, int r, uint32_t steps, uint8_t flag) {
  const size_t o = (size_t)(M.y0 + r / M.tw) * M.cam->W + (M.x0 + r % M.tw);
  M.out->depth[o] = INFINITY;
  M.out->normal[3 * o] = 0.f;
  M.out->normal[3 * o + 1] = 0.f;
  M.out->normal[3 * o + 2] = 0.f;
  M.out->evals[o] = steps;
  M.out->flags[o] = flag;
}

// Appends the rays of the set lanes to a shared list (warp-aggregated).
__device__ __forceinline__ void append_rays(bool want, int r, uint16_t *list, int *counter) {
  const uint32_t m = __ballot_sync(0xFFFFFFFFu, want);
  if (!m) return;
  int base = 0;
  const int lane = threadIdx.x & 31;
  if (lane == __ffs(m) - 1) base = atomicAdd(counter, __popc(m));
  base = __shfl_sync(0xFFFFFFFFu, base, __ffs(m) - 1);
  if (want) list[base + __popc(m & lanemask_lt())] = (uint16_t)r;
}

// ---- tail sharing between the warps of a tile ----------------------------------
// A warp that is down to a few rays of a subfrustum keeps one and hands the
// others to a shared queue (state saved per ray in shared memory); warps
// without rays pop them instead of waiting at the end of the subfrustum.  A
// ray's trajectory does not depend on the warp that steps it.  Entries are
// (tag << 32) | ray with a tag unique per subfrustum of the CTA, so a popper
// can wait for the pusher's store; every wait is bounded.
constexpr uint32_t kIdleSpinLimit = 1u << 22;
constexpr uint32_t kEntrySpinLimit = 1u << 16;

__device__ __forceinline__ int tq_pop(unsigned long long *tq, int *tail, int *head, uint32_t tag, int cap,
                                      uint32_t &err) {
  const int t = *(volatile int *)tail;
  const int h = *(volatile int *)head;
  if (h >= t || h >= cap) return -1;
  if (atomicCAS(head, h, h + 1) != h) return -1;
  for (uint32_t it = 0; it < kEntrySpinLimit; ++it) {
    const unsigned long long e = *(volatile unsigned long long *)(tq + h);
    if ((uint32_t)(e >> 32) == tag) {
      __threadfence_block();
      return (int)(uint32_t)(e & 0xFFFFFFFFull);
    }
    __nanosleep(20);
  }
  err |= ST_STATUS_WAIT;
  return -1;
}

// ---- splitting a long-running tile across CTAs ----------------------------------
// A handful of tiles (grazing rays near silhouettes: many steps over large
// views) can take longer than the whole rest of the frame.  A CTA whose tile
// is still tracing after L.split_cycles publishes, at a subfrustum boundary,
// the state of the tile's pending rays (depth reached, steps) as a split
// record of P parts: part p holds the pending rays i = p (mod P).  It keeps
// part 0; CTAs looking for work claim the other parts before new tiles,
// replay the tile's segmentation up to the resume subfrustum (it depends on
// the A-buffer list only) and trace their rays from there.  A ray's
// trajectory does not depend on the CTA that steps it, so the output is the
// same.  Nothing waits on another CTA: a CTA that pushed a record claims its
// unclaimed parts itself before it leaves, and an idle CTA only polls
// (boundedly) while whole tiles are still being traced.
//
// Split area (words): [0] records taken, [1] no open part below this record,
// [2] CTAs tracing a whole tile, [3] unused, [4, 4 + cap) parts P of record r
// (0 until published), [4 + cap, 4 + 2 cap) parts of record r claimed by
// other CTAs; then the records (split_rec_words each): [0] global tile,
// [1] subfrustum to resume at, [2] pending rays n, [3] unused,
// [4, 4 + rays) pending ray ids, then depth reached and steps | status by
// ray id (rays = max_tile_rays).
constexpr int kSplitMinRays = 8;    // pending rays per part at least
constexpr int kSplitMaxParts = 16;
constexpr int kHeavyParts = 8;      // parts of a tile split before its first subfrustum
constexpr uint32_t kSplitListBudget = 4096;   // parts x A-buffer list length at most
constexpr uint32_t kSplitIdleSpins = 1u << 21;   // polls of an idle CTA (x ~1 us)

__device__ __forceinline__ uint32_t *split_record(const TraceLaunch &L, uint32_t r) {
  return L.split + 4 + 2 * (size_t)L.split_cap + (size_t)r * split_rec_words(L.max_tile_rays);
}

// One thread, no waiting: claims an unclaimed part of a published split
// record (tiles split before their first subfrustum are open while whole
// tiles remain; CTAs take their parts first).  Returns the part's global
// tile with *part >= 1 and *rec, or 0xFFFFFFFF when no part is open now.
__device__ __forceinline__ uint32_t try_part(const TraceLaunch &L, uint32_t *rec, int *part) {
  uint32_t *hdr = L.split;
  uint32_t *parts = hdr + 4, *claimed = hdr + 4 + L.split_cap;
  const uint32_t n = min(*(volatile uint32_t *)&hdr[0], L.split_cap);
  bool prefix = true;   // records below r are published and fully claimed
  for (uint32_t r = *(volatile uint32_t *)&hdr[1]; r < n; ++r) {
    const uint32_t P = *(volatile uint32_t *)&parts[r];
    if (P > 1 && *(volatile uint32_t *)&claimed[r] + 1 < P) {
      const uint32_t c = atomicAdd(&claimed[r], 1u);
      if (c + 1 < P) {
        __threadfence();   // the record's contents were published before P
        *rec = r;
        *part = (int)c + 1;
        return __ldcg(split_record(L, r));
      }
    }
    if (P == 0 || *(volatile uint32_t *)&claimed[r] + 1 < P) prefix = false;
    if (prefix) atomicMax(&hdr[1], r + 1);
  }
  return 0xFFFFFFFFu;
}

// One thread: claims an unclaimed part of a split record, polling while
// whole tiles are still being traced (they may split; a record published
// before the last of them ended is visible to one more scan).  Returns the
// part's global tile with *part >= 1 and *rec, or 0xFFFFFFFF: no work left.
__device__ __forceinline__ uint32_t next_part(const TraceLaunch &L, uint32_t *rec, int *part) {
  uint32_t *hdr = L.split;
  uint32_t *parts = hdr + 4, *claimed = hdr + 4 + L.split_cap;
  bool last = false;
  for (uint32_t spins = 0;; ++spins) {
    const uint32_t n = min(*(volatile uint32_t *)&hdr[0], L.split_cap);
    uint32_t r = *(volatile uint32_t *)&hdr[1];
    bool prefix = true;   // records below r are published and fully claimed
    for (; r < n; ++r) {
      const uint32_t P = *(volatile uint32_t *)&parts[r];
      if (P > 1 && *(volatile uint32_t *)&claimed[r] + 1 < P) {
        const uint32_t c = atomicAdd(&claimed[r], 1u);
        if (c + 1 < P) {
          __threadfence();   // the record's contents were published before P
          *rec = r;
          *part = (int)c + 1;
          return __ldcg(split_record(L, r));
        }
      }
      if (P == 0 || *(volatile uint32_t *)&claimed[r] + 1 < P) prefix = false;
      if (prefix) atomicMax(&hdr[1], r + 1);
    }
    if (last) return 0xFFFFFFFFu;
    if (*(volatile uint32_t *)&hdr[2] == 0u || spins >= (L.split_spins ? L.split_spins : kSplitIdleSpins)) {
      __threadfence();
      last = true;
      continue;
    }
    __nanosleep(1000);
  }
}

// Returns the number of live ray-steps taken by this lane.  `wvals` is the
// warp's evaluation-stack memory viewed as floats (tail mode scratch).
struct LearnCtx {      // learned step / recording context of a subfrustum
  MlpSmem W;
  uint32_t list_len;
  const TraceLaunch *L;
  unsigned long long *diag;   // tile diagnostics (shared, null when off): lockstep
                              // iterations, live slots over them, tail evaluations,
                              // refinement passes, live lanes over them
  float4 *stage;              // this warp's record stage (staged instances)
};

template <int MODE, int kFam, bool kStaged, bool kCta>
__device__ __forceinline__ uint32_t march_sub(const MarchCtx &M, const CtaWork &C, const RecSrc &src, const SubInfo &inf,
                              const uint32_t *view, const uint2 *ops, const int *lvl_off, const uint16_t *alive_in,
                              int n_in, int *q_head, uint16_t *alive_out, int *n_out, uint16_t *hits, int &n_hits,
                              float2 *stk_lane, float *wvals, int vals_cap, uint64_t &c_rej,
                              const LearnCtx &LC, int *tq_tail, int *tq_head, int *n_done, int *n_idle,
                              uint32_t tag, uint32_t &c_err, int cta_slot) {
  constexpr bool kShare = MODE != ST_STEP_RECORD;
  // CTA-split evaluation (staged instances; see build_cta_split): once the
  // subfrustum's pending list is drained and at most kCtaMaxRays of its rays
  // are unfinished, the first warp to notice (holding rays itself) becomes
  // the owner: the others hand it their rays through the tail queue and
  // help.  Each pass the owner publishes its points, every warp evaluates its
  // segment of the view for them (named barrier 1 before, 2 after), and the
  // owner evaluates the top program and steps the rays.  A warp can only
  // leave the subfrustum when all of its rays are finished, which cannot
  // happen before the owner's request is visible, so every warp joins; the
  // joins and the go are still bounded waits, and a request that runs out is
  // abandoned (CAS on the flag) before any barrier is taken.
  constexpr bool kCtaOk = kStaged && kShare && kCta;
  int cta = 0;   // 0 normal, 1 owner, 2 helper
  CtaSync *const cs = &s_ctash.sync[cta_slot];
  const bool cta_ok = kCtaOk && s_ctash.info[cs->vb].n_top > 0;
  if (kCtaOk && threadIdx.x == 0) atomicExch(&cs->w0in, 1);
  uint32_t idle_spins = 0;
  const uint32_t idle_limit = LC.L->idle_spins ? LC.L->idle_spins : kIdleSpinLimit;
  bool idle = false;   // this warp is registered in *n_idle (waiting for handed-over rays)
  uint32_t rejected = 0;
  const int lane = threadIdx.x & 31;
  const float eps = M.tp->eps;
  const float z_begin = inf.z_begin, z_end = inf.z_end;
  int ray[kR];
  float z[kR], d[kR][3], inv_ld[kR];
  uint32_t steps[kR];
  // Relaxed stepping state (Sec. 10, sphere tracing with over-relaxation): the
  // surface-free radius rp of the previous point, the last step length dzp
  // (0: no previous point in this subfrustum; a plain step has dzp = rp and
  // can never be rejected), the plain-step position zf = previous point + rp
  // to fall back to, and a stored surface-free sphere (zs, rs; rs < 0:
  // none); relaxation is off from a rejected step until that sphere is crossed.
  float rp[kR], dzp[kR], zf[kR], zs[kR], rs[kR];
  uint32_t relax_off = 0u;
  // Field value at the previous point (learned features); recording mode
  // also keeps the value two points back, the step between them and how
  // many consecutive plain steps this subfrustum has seen (0..2).
  float fpv[kR], fpp[kR], dpp[kR];
  int hv[kR];
#pragma unroll
  for (int s = 0; s < kR; ++s) {
    ray[s] = -1; z[s] = 0.f; inv_ld[s] = 0.f; steps[s] = 0; d[s][0] = d[s][1] = d[s][2] = 0.f;
    rp[s] = dzp[s] = zf[s] = 0.f; zs[s] = 0.f; rs[s] = -1.f;
    fpv[s] = fpp[s] = dpp[s] = 0.f; hv[s] = 0;
  }
  const float inv_l = 1.f / M.tp->lipschitz;
  // Per-subfrustum features of the learned step (see step_features).
  const float feat_prim = log2f(1.f + (float)inf.n_prim) * 0.125f;
  const float feat_len = log2f(1.f + (float)LC.list_len) * 0.125f;
  const float omega_c = MODE == ST_STEP_OVERRELAX || MODE == ST_STEP_CROSSING ? M.tp->omega : 1.f;
  // Shortest step of ST_STEP_CROSSING times L: with inv_ld = 1 / (L |d|) the
  // step along the ray parameter is min_l x inv_ld.
  const float min_l = MODE == ST_STEP_CROSSING ? mul_(M.tp->min_step, M.tp->lipschitz) : 0.f;
  bool drained = false;
  uint32_t live_steps = 0;
  SmemStack2 stk{stk_lane};
  // Tail mode pays one parallel pass per remaining ray instead of one
  // lockstep pass over the whole view for all rays.
  const bool tail_ok = inf.n_lvl > 0 && inf.n_view <= vals_cap;
  const int tail_cost = ((inf.n_view + 1) / 2 + 31) / 32 + 2 * inf.n_lvl + 2;   // (n primitives: 2n - 1 nodes)

  // One step of slot s with field value fs: hit / leave the subfrustum /
  // step cap / advance.  Records hits and hand-overs in shared memory.
  auto leave_or_cap = [&](int s, bool &exit) {
    if (z[s] >= z_end) {
      exit = true;
      C.ray_z[ray[s]] = z_end;
      C.ray_st[ray[s]] = steps[s];
    } else if ((int)steps[s] >= (MODE == ST_STEP_CROSSING ? kStepFieldMax : M.tp->max_steps)) {
      C.ray_st[ray[s]] = steps[s] | (R_UNCONV << 24);
      write_miss(M, ray[s], steps[s], 2);
      ray[s] = -1;
    }
  };
  // One step of slot s with field value fs and proposed relaxation factor
  // om_prop: rejection test of the previous relaxed step, hit, reuse of a
  // stored sphere, then the (possibly relaxed) step f / (L |d|) x omega.
  auto step_slot = [&](int s, float fs, float om_prop, bool &hit, bool &exit) {
    hit = exit = false;
    if (ray[s] < 0) return;
    ++steps[s];
    ++live_steps;
    const uint32_t bit = 1u << s;
    if (MODE == ST_STEP_RECORD) {
      // Record the previous plain step (its features and the label that
      // the value reached now gives it), then remember this point.
      const int r = ray[s];
      const uint32_t pix = (uint32_t)(M.y0 + r / M.tw) * (uint32_t)M.cam->W + (uint32_t)(M.x0 + r % M.tw);
      if (hv[s] >= 1 && (pix % (uint32_t)LC.L->rec_stride) == 0u) {
        float x[6];
        step_features(fpv[s], fpp[s], dpp[s], hv[s] >= 2, steps[s] - 1, inf.n_prim, LC.list_len, inv_l, x);
        const uint32_t slot = atomicAdd(LC.L->rec_count, 1u);
        if (slot < LC.L->rec_cap) {
          float4 *dst = reinterpret_cast<float4 *>(LC.L->records + (size_t)slot * 8);
          dst[0] = make_float4(x[0], x[1], x[2], x[3]);
          dst[1] = make_float4(x[4], x[5], step_label(fpv[s], fs), 0.f);
        }
      }
      fpp[s] = fpv[s];
      dpp[s] = mul_(fs, inv_l);   // the plain step taken from this point, in distance units
      fpv[s] = fs;
      hv[s] = hv[s] < 2 ? hv[s] + 1 : 2;
    }
    // Explicit rounding throughout: the two slots are separate unrolled
    // copies of this code, and a ray may move between slots and warps.
    const float r = mul_(fabsf(fs), inv_ld[s]);   // surface-free radius along the ray
    if (MODE != ST_STEP_PLAIN && MODE != ST_STEP_RECORD && add_(r, rp[s]) < dzp[s]) {
      // The unbounding spheres of the last two points do not overlap: the
      // relaxed step may have skipped a crossing.  Keep the landing sphere,
      // return to the previous point and take the plain step from there.
      zs[s] = z[s];
      rs[s] = r;
      if (MODE == ST_STEP_CROSSING && fs <= 0.f) {
        // Landed inside the solid: a crossing lies before this point, so
        // plain steps go on until they bracket it (a sphere that is never
        // reached keeps relaxation off, and none is jumped over).
        zs[s] = __int_as_float(0x7f800000);
        rs[s] = 0.f;
      }
      z[s] = zf[s];
      dzp[s] = 0.f;
      relax_off |= bit;
      ++rejected;
      if (z[s] >= sub_(zs[s], rs[s])) {
        z[s] = add_(zs[s], rs[s]);
        rs[s] = -1.f;
        relax_off &= ~bit;
      }
      leave_or_cap(s, exit);
      return;
    }
    if (MODE == ST_STEP_CROSSING ? fs <= 0.f : fs <= eps) {
      hit = true;
      C.ray_z[ray[s]] = z[s];
      C.ray_st[ray[s]] = steps[s] | (R_HIT << 24);
      return;
    }
    if (MODE == ST_STEP_PLAIN || MODE == ST_STEP_RECORD) {
      z[s] = add_(z[s], r);
      leave_or_cap(s, exit);
      return;
    }
    fpv[s] = fs;   // value at the point the (possibly relaxed) step starts from
    float om = (relax_off & bit) ? 1.f : om_prop;
    float dz = mul_(om, r);
    if (om > 1.f && add_(z[s], dz) >= z_end) { om = 1.f; dz = r; }   // relaxed steps never cross z_end
    float dz_plain = r;
    if (MODE == ST_STEP_CROSSING) {
      // Shortest step: it may cross the surface (by less than min_step), and
      // the sign test at the next sample detects the crossing; a step that
      // the minimum lengthened is not a relaxed step and is never rejected.
      const float h = mul_(min_l, inv_ld[s]);
      if (dz <= h) { dz = h; om = 1.f; }
      dz_plain = fmaxf(r, h);
    }
    zf[s] = add_(z[s], dz_plain);
    rp[s] = r;
    dzp[s] = (MODE == ST_STEP_CROSSING && om <= 1.f) ? r : dz;
    z[s] = add_(z[s], dz);
    if ((relax_off & bit) && rs[s] >= 0.f && z[s] >= sub_(zs[s], rs[s])) {
      // Plain stepping reached the stored surface-free sphere: cross it.
      z[s] = fmaxf(z[s], add_(zs[s], rs[s]));
      rs[s] = -1.f;
      relax_off &= ~bit;
      dzp[s] = 0.f;
    }
    leave_or_cap(s, exit);
  };
  auto retire = [&](int s, bool hit, bool exit) {   // warp-collective
    const uint32_t hm = __ballot_sync(0xFFFFFFFFu, hit);
    if (hit) hits[n_hits + __popc(hm & lanemask_lt())] = (uint16_t)ray[s];
    n_hits += __popc(hm);
    append_rays(exit, ray[s], alive_out, n_out);
    if (hit || exit) ray[s] = -1;
  };

  // Hands every live ray of this warp to the tail queue (state saved by ray).
  auto give_all = [&]() {
#pragma unroll
    for (int s = 0; s < kR; ++s) {
      const bool give = ray[s] >= 0;
      const uint32_t gm = __ballot_sync(0xFFFFFFFFu, give);
      if (!gm) continue;
      if (give) {
        const int r = ray[s];
        C.ray_z[r] = z[s];
        C.ray_st[r] = steps[s];
        C.rs4[r] = make_float4(rp[s], dzp[s], zf[s], zs[s]);
        C.rs2[r] = make_float2(rs[s], fpv[s]);
      }
      __threadfence_block();
      int base = 0;
      if (lane == __ffs(gm) - 1) base = atomicAdd(tq_tail, __popc(gm));
      base = __shfl_sync(0xFFFFFFFFu, base, __ffs(gm) - 1);
      const int idx = base + __popc(gm & lanemask_lt());
      if (give && idx < tq_cap(*LC.L)) {
        *(volatile unsigned long long *)(C.tq + idx) = ((unsigned long long)tag << 32) | (uint32_t)ray[s];
        ray[s] = -1;
      }
    }
  };

  for (;;) {
    int n_live = 0;
    if (kCtaOk && cta == 2) {
      // ---- CTA-split helper: wait for the owner's points or its end ----
      cta_bar(1);
      if (*(volatile int *)&cs->cmd == kCtaDone) break;
    } else {
    if (kCtaOk && cta_ok && cta == 0) {
      // ---- CTA-split request and joins ----
      int st = 0;
      if (lane == 0) st = *(volatile int *)&cs->flag;
      st = __shfl_sync(0xFFFFFFFFu, st, 0);
      if (st == 0 && drained && *(volatile int *)&cs->w0in &&
          __any_sync(0xFFFFFFFFu, ray[0] >= 0 || ray[1] >= 0)) {
        int won = 0;
        if (lane == 0) {
          if (n_in - *(volatile int *)n_done <= kCtaMaxRays) won = atomicCAS(&cs->flag, 0, 1) == 0;
          st = *(volatile int *)&cs->flag;
        }
        won = __shfl_sync(0xFFFFFFFFu, won, 0);
        st = __shfl_sync(0xFFFFFFFFu, st, 0);
        if (won) cta = 1;
      }
      if (cta == 0 && st == 1) {
        // join: hand every ray to the owner, then wait for its go
        give_all();
        if (idle && lane == 0) atomicSub(n_idle, 1);
        idle = false;
        __threadfence_block();
        int g = 0;
        if (lane == 0) {
          atomicAdd(&cs->join, 1);
          for (uint32_t it = 0;; ++it) {
            g = *(volatile int *)&cs->flag;
            if (g != 1) break;
            if (it >= idle_limit) {
              g = atomicCAS(&cs->flag, 1, 3);
              if (g == 1) { g = 3; c_err |= ST_STATUS_WAIT; }
              break;
            }
            __nanosleep(64);
          }
        }
        g = __shfl_sync(0xFFFFFFFFu, g, 0);
        if (g == 2) {
          cta = 2;
          continue;
        }
        // abandoned: this warp carries on without rays (tail sharing as usual)
      }
      if (cta == 1) {
        // owner: wait until every other warp has handed its rays over
        int g = 0;
        if (lane == 0) {
          for (uint32_t it = 0;; ++it) {
            if (*(volatile int *)&cs->join >= kWarps - 1) {
              g = atomicCAS(&cs->flag, 1, 2);
              break;
            }
            if (*(volatile int *)&cs->flag != 1) {   // a helper's bound ran out
              g = 3;
              break;
            }
            if (it >= idle_limit) {
              atomicCAS(&cs->flag, 1, 3);   // abandoned either way (3 already, or now)
              g = 3;
              c_err |= ST_STATUS_WAIT;
              break;
            }
            __nanosleep(64);
          }
        }
        g = __shfl_sync(0xFFFFFFFFu, g, 0);
        if (g != 1) cta = 0;   // abandoned (by a helper's or this warp's bound)
        __threadfence_block();
      }
    }
    // ---- refill empty slots from the tile's pending-ray list ----
    uint32_t need_m[kR];
    int n_need = 0;
#pragma unroll
    for (int s = 0; s < kR; ++s) {
      need_m[s] = __ballot_sync(0xFFFFFFFFu, ray[s] < 0);
      n_need += __popc(need_m[s]);
    }
    if (kCtaOk && cta == 1 && n_need) {
      // owner: the handed-over rays, as many as there are free slots
#pragma unroll
      for (int s = 0; s < kR; ++s) {
        if (!need_m[s]) continue;
        int h = 0, t = 0;
        if (lane == 0) { h = *(volatile int *)tq_head; t = *(volatile int *)tq_tail; }
        h = __shfl_sync(0xFFFFFFFFu, h, 0);
        t = __shfl_sync(0xFFFFFFFFu, t, 0);
        const int take = min(__popc(need_m[s]), min(t, tq_cap(*LC.L)) - h);
        if (take <= 0) continue;
        if (lane == 0) atomicAdd(tq_head, take);
        const int rank = __popc(need_m[s] & lanemask_lt());
        if (ray[s] < 0 && rank < take) {
          int got = -1;
          for (uint32_t it = 0; it < kEntrySpinLimit; ++it) {
            const unsigned long long e = *(volatile unsigned long long *)(C.tq + h + rank);
            if ((uint32_t)(e >> 32) == tag) {
              got = (int)(uint32_t)(e & 0xFFFFFFFFull);
              break;
            }
            __nanosleep(20);
          }
          if (got < 0) {
            c_err |= ST_STATUS_WAIT;
          } else {
            __threadfence_block();
            ray[s] = got;
            load_ray(M, C, got, z_begin, z[s], steps[s], d[s], inv_ld[s]);
            const float4 a = C.rs4[got];
            const float2 b = C.rs2[got];
            rp[s] = a.x; dzp[s] = a.y; zf[s] = a.z; zs[s] = a.w;
            rs[s] = b.x; fpv[s] = b.y;
            relax_off = rs[s] >= 0.f ? (relax_off | (1u << s)) : (relax_off & ~(1u << s));
            hv[s] = 0;
          }
        }
      }
    }
    if (cta == 0 && n_need && !drained) {
      // A warp takes at most its share of the subfrustum's rays at a time,
      // so that short lists spread over the warps of the CTA.
      const int take = min(n_need, (n_in + kWarps - 1) / kWarps);
      int base = 0;
      if (lane == 0) base = atomicAdd(q_head, take);
      base = __shfl_sync(0xFFFFFFFFu, base, 0);
      if (base + take >= n_in) drained = true;
      int off = 0;
#pragma unroll
      for (int s = 0; s < kR; ++s) {
        const int idx = off + __popc(need_m[s] & lanemask_lt());
        const int rk = base + idx;
        if (ray[s] < 0 && idx < take && rk < n_in) {
          ray[s] = alive_in[rk];
          load_ray(M, C, ray[s], z_begin, z[s], steps[s], d[s], inv_ld[s]);
          dzp[s] = 0.f;
          rp[s] = 0.f;
          rs[s] = -1.f;
          relax_off &= ~(1u << s);
          hv[s] = 0;
        }
        off += __popc(need_m[s]);
      }
    }
    if (kShare && cta == 0 && drained && !__any_sync(0xFFFFFFFFu, ray[0] >= 0 || ray[1] >= 0)) {
      // Out of rays: take one handed over by another warp.
      if (!idle && lane == 0) atomicAdd(n_idle, 1);
      idle = true;
      int got = -1;
      if (lane == 0) got = tq_pop(C.tq, tq_tail, tq_head, tag, tq_cap(*LC.L), c_err);
      got = __shfl_sync(0xFFFFFFFFu, got, 0);
      if (got >= 0) {
        if (lane == 0) atomicSub(n_idle, 1);
        idle = false;
      }
      if (got >= 0 && lane == 0) {
        ray[0] = got;
        load_ray(M, C, got, z_begin, z[0], steps[0], d[0], inv_ld[0]);
        const float4 a = C.rs4[got];
        const float2 b = C.rs2[got];
        rp[0] = a.x; dzp[0] = a.y; zf[0] = a.z; zs[0] = a.w;
        rs[0] = b.x; fpv[0] = b.y;
        relax_off = rs[0] >= 0.f ? (relax_off | 1u) : (relax_off & ~1u);
        hv[0] = 0;
      }
    }
#pragma unroll
    for (int s = 0; s < kR; ++s) n_live += __popc(__ballot_sync(0xFFFFFFFFu, ray[s] >= 0));
    if (n_live == 0) {
      if (!kShare) break;
      if (kCtaOk && cta == 1) {
        // owner: every ray is finished; release the helpers
        if (lane == 0) {
          *(volatile int *)&cs->own = threadIdx.x >> 5;
          *(volatile int *)&cs->nh = n_hits;
          *(volatile int *)&cs->cmd = kCtaDone;
        }
        __threadfence_block();
        cta_bar(1);
        break;
      }
      // Every ray of the subfrustum finished?  Else wait for handed-over rays.
      if (*(volatile int *)n_done >= n_in || ++idle_spins > idle_limit) {
        if (idle_spins > idle_limit) c_err |= ST_STATUS_WAIT;
        if (idle && lane == 0) atomicSub(n_idle, 1);
        break;
      }
      __nanosleep(64);
      continue;
    }
    }

    float f[kR];
    const bool tail_now = cta == 0 && drained && tail_ok && n_live * tail_cost < inf.n_view;
    if (LC.diag && lane == 0 && cta != 2) {
      if (cta == 1) {
        atomicAdd(&LC.diag[5], 1ull);
        atomicAdd(&LC.diag[6], (unsigned long long)n_live);
      } else if (tail_now) {
        atomicAdd(&LC.diag[2], (unsigned long long)n_live);
      } else {
        atomicAdd(&LC.diag[0], 1ull);
        atomicAdd(&LC.diag[1], (unsigned long long)n_live);
      }
    }
    if (tail_now) {
      int n_give = 0;
      if (kShare && n_live > 1) n_give = min(n_live - 1, *(volatile int *)n_idle);
      n_give = __shfl_sync(0xFFFFFFFFu, n_give, 0);
      if (n_give > 0) {
        // Keep the first live ray, hand up to one ray per idle warp over.
        const uint32_t m0 = __ballot_sync(0xFFFFFFFFu, ray[0] >= 0), m1 = __ballot_sync(0xFFFFFFFFu, ray[1] >= 0);
        const int keep_s = m0 ? 0 : 1;
        const int keep_l = __ffs(m0 ? m0 : m1) - 1;
        int given = 0;
#pragma unroll
        for (int s = 0; s < kR; ++s) {
          const bool cand = ray[s] >= 0 && !(s == keep_s && lane == keep_l);
          const uint32_t cm = __ballot_sync(0xFFFFFFFFu, cand);
          const bool give = cand && given + __popc(cm & lanemask_lt()) < n_give;
          given += __popc(cm);
          const uint32_t gm = __ballot_sync(0xFFFFFFFFu, give);
          if (!gm) continue;
          if (give) {
            const int r = ray[s];
            C.ray_z[r] = z[s];
            C.ray_st[r] = steps[s];
            C.rs4[r] = make_float4(rp[s], dzp[s], zf[s], zs[s]);
            C.rs2[r] = make_float2(rs[s], fpv[s]);
          }
          __threadfence_block();
          int base = 0;
          if (lane == __ffs(gm) - 1) base = atomicAdd(tq_tail, __popc(gm));
          base = __shfl_sync(0xFFFFFFFFu, base, __ffs(gm) - 1);
          const int idx = base + __popc(gm & lanemask_lt());
          if (give && idx < tq_cap(*LC.L)) {
            *(volatile unsigned long long *)(C.tq + idx) = ((unsigned long long)tag << 32) | (uint32_t)ray[s];
            ray[s] = -1;
          }
        }
      }
      // ---- tail: evaluate each remaining ray with the whole warp; the
      // owner lane receives its ray's value ----
#pragma unroll
      for (int s = 0; s < kR; ++s) {
        f[s] = 0.f;
        uint32_t m = __ballot_sync(0xFFFFFFFFu, ray[s] >= 0);
        while (m) {
          const int owner = __ffs(m) - 1;
          m &= m - 1;
          const float zz = __shfl_sync(0xFFFFFFFFu, z[s], owner);
          const float pt[3] = {fma_(zz, __shfl_sync(0xFFFFFFFFu, d[s][0], owner), M.cam->o[0]),
                               fma_(zz, __shfl_sync(0xFFFFFFFFu, d[s][1], owner), M.cam->o[1]),
                               fma_(zz, __shfl_sync(0xFFFFFFFFu, d[s][2], owner), M.cam->o[2])};
          const float fv = tail_eval<kFam>(view, inf.n_view, ops, lvl_off, inf.n_lvl, src, pt, wvals);
          if (lane == owner) f[s] = fv;
        }
      }
    } else {
      // ---- one lockstep field evaluation per slot (Algorithm 3 over the view) ----
      // At most 32 rays left but some lane holds two: lanes with two rays hand
      // their second ray to lanes with none (warp shuffles), so that one
      // evaluation chain per lane suffices.  (Not in a CTA-split pass: its
      // helpers evaluate pairs.)
      if (cta == 0) {
        const uint32_t two = __ballot_sync(0xFFFFFFFFu, ray[0] >= 0 && ray[1] >= 0);
        const uint32_t none = __ballot_sync(0xFFFFFFFFu, ray[0] < 0 && ray[1] < 0);
        if (two && n_live <= 32) {
          const int rank_t = __popc(none & lanemask_lt());
          const bool take = ((none >> lane) & 1u) && rank_t < __popc(two);
          const int src_l = take ? kth_set_bit(two, rank_t) : lane;
          const bool give = ((two >> lane) & 1u) && __popc(two & lanemask_lt()) < __popc(none);
          const int r_r = __shfl_sync(0xFFFFFFFFu, ray[1], src_l);
          const float z_r = __shfl_sync(0xFFFFFFFFu, z[1], src_l);
          const float d0_r = __shfl_sync(0xFFFFFFFFu, d[1][0], src_l);
          const float d1_r = __shfl_sync(0xFFFFFFFFu, d[1][1], src_l);
          const float d2_r = __shfl_sync(0xFFFFFFFFu, d[1][2], src_l);
          const float il_r = __shfl_sync(0xFFFFFFFFu, inv_ld[1], src_l);
          const uint32_t st_r = __shfl_sync(0xFFFFFFFFu, steps[1], src_l);
          const float rp_r = __shfl_sync(0xFFFFFFFFu, rp[1], src_l);
          const float dzp_r = __shfl_sync(0xFFFFFFFFu, dzp[1], src_l);
          const float zf_r = __shfl_sync(0xFFFFFFFFu, zf[1], src_l);
          const float zs_r = __shfl_sync(0xFFFFFFFFu, zs[1], src_l);
          const float rs_r = __shfl_sync(0xFFFFFFFFu, rs[1], src_l);
          const float fpv_r = __shfl_sync(0xFFFFFFFFu, fpv[1], src_l);
          const float fpp_r = __shfl_sync(0xFFFFFFFFu, fpp[1], src_l);
          const float dpp_r = __shfl_sync(0xFFFFFFFFu, dpp[1], src_l);
          const int hv_r = __shfl_sync(0xFFFFFFFFu, hv[1], src_l);
          const uint32_t ro_r = __shfl_sync(0xFFFFFFFFu, (relax_off >> 1) & 1u, src_l);
          if (take) {
            ray[0] = r_r; z[0] = z_r; d[0][0] = d0_r; d[0][1] = d1_r; d[0][2] = d2_r; inv_ld[0] = il_r;
            steps[0] = st_r; rp[0] = rp_r; dzp[0] = dzp_r; zf[0] = zf_r; zs[0] = zs_r; rs[0] = rs_r;
            fpv[0] = fpv_r; fpp[0] = fpp_r; dpp[0] = dpp_r; hv[0] = hv_r;
            relax_off = (relax_off & ~1u) | ro_r;
          }
          if (give) {
            ray[1] = -1;
            relax_off &= ~2u;
          }
        }
      }
      // A lane whose first slot is empty takes its second slot's ray; when no
      // lane has a second ray left, one evaluation chain per lane suffices.
      const bool mv = cta == 0 && ray[0] < 0 && ray[1] >= 0;
      if (mv) {
        ray[0] = ray[1]; z[0] = z[1]; inv_ld[0] = inv_ld[1]; steps[0] = steps[1];
        d[0][0] = d[1][0]; d[0][1] = d[1][1]; d[0][2] = d[1][2];
        rp[0] = rp[1]; dzp[0] = dzp[1]; zf[0] = zf[1]; zs[0] = zs[1]; rs[0] = rs[1];
        fpv[0] = fpv[1]; fpp[0] = fpp[1]; dpp[0] = dpp[1]; hv[0] = hv[1];
        relax_off = (relax_off & ~3u) | ((relax_off >> 1) & 1u);
        ray[1] = -1;
      }
      // (The learned step's instances and those with the CTA split evaluate
      // pairs only: a pair with one live ray issues the same instructions as
      // the single chain, and one interpreter instance less leaves the
      // learned kernel's code and registers to the rest.  Measured on B300:
      // learned 1080p 4.26 -> 3.98 ms, six families 10.6 -> 9.8 ms; the other
      // step modes are 3-5 % faster with the single chain kept.)
      if (!kCtaOk && MODE != ST_STEP_LEARNED && !__any_sync(0xFFFFFFFFu, ray[1] >= 0)) {
        float p1[1][3] = {{fma_(z[0], d[0][0], M.cam->o[0]), fma_(z[0], d[0][1], M.cam->o[1]),
                           fma_(z[0], d[0][2], M.cam->o[2])}};
        float f1[1];
        SmemStack1 stk1{stk.base};
        if (kStaged)
          eval_view_staged<1, float, SmemStack1, kFam>(view, inf.n_view, src, p1, f1, stk1, LC.stage);
        else
          eval_view_r<1, float, SmemStack1, kFam>(view, inf.n_view, src, p1, f1, stk1);
        f[0] = f1[0];
        f[1] = 0.f;
      } else {
        // the two slots' points as one pair: paired FP32 instructions
        F2 p2[1][3];
        if (cta != 2) {
          const F2 zz = F2(make_float2(z[0], z[1]));
#pragma unroll
          for (int k = 0; k < 3; ++k) p2[0][k] = fma_(zz, F2(make_float2(d[0][k], d[1][k])), M.cam->o[k]);
        }
        F2 f2[1];
        using Stk2 = std::conditional_t<kCtaOk, SmemStackF2Cta, SmemStackF2>;
        Stk2 stk2{stk.base};
        const uint32_t *ev_view = view;
        int ev_n = inf.n_view;
        RecSrc ev_src = src;
        if (kCtaOk && cta != 0) {
          // CTA-split pass: the owner publishes its points; every warp
          // evaluates its segment, storing its forest roots' values
          const int warp_id = threadIdx.x >> 5;
          const CtaInfo *ci = &s_ctash.info[cs->vb];
          float4 *crec = s_ctash.crec;
          float2 *cpts = reinterpret_cast<float2 *>(crec + 2 * kCtaTopMax + 16 * kCtaOutMax);
          if (cta == 1) {
#pragma unroll
            for (int k = 0; k < 3; ++k) __stcg(cpts + k * 32 + lane, p2[0][k].v);
            if (lane == 0) *(volatile int *)&cs->cmd = 1;
            __threadfence_block();
            cta_bar(1);
          } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) p2[0][k] = F2(__ldcg(cpts + k * 32 + lane));
          }
          ev_view = s_ctash.cseg[cs->vb] + ci->off[warp_id];
          ev_n = ci->len[warp_id];
          if constexpr (kCtaOk) {
            stk2.xout = reinterpret_cast<float2 *>(crec + 2 * kCtaTopMax) + (size_t)ci->slot[warp_id] * 32;
            stk2.xn = 0;
          }
        }
        for (int ph = 0;; ++ph) {
          if (kStaged)
            eval_view_staged<1, F2, Stk2, kFam>(ev_view, ev_n, ev_src, p2, f2, stk2, LC.stage);
          else
            eval_view_r<1, F2, Stk2, kFam>(view, inf.n_view, src, p2, f2, stk2);
          if (!kCtaOk || cta == 0 || ph > 0) break;
          // every segment's values are stored: the owner combines them
          __threadfence_block();
          cta_bar(2);
          if (cta == 2) break;
          ev_view = s_ctash.ctop[cs->vb];
          ev_n = s_ctash.info[cs->vb].n_top;
          ev_src = RecSrc{s_ctash.crec, src.dc};
        }
        f[0] = f2[0].v.x;
        f[1] = f2[0].v.y;
      }
    }
    if (kCtaOk && cta == 2) continue;   // helpers: the owner steps the rays
    float om[kR];
#pragma unroll
    for (int s = 0; s < kR; ++s) om[s] = omega_c;
    if (MODE == ST_STEP_LEARNED) {
      // One BF16 tensor-core MLP pass over the warp's live slots (the
      // evaluation stack memory is free again and holds the fragments).
      // The factor of a step depends on its ray's state alone, whichever
      // evaluation path produced f.
      float x[2][6];
      uint32_t live = 0u;
#pragma unroll
      for (int s = 0; s < kR; ++s) {
        const float dist = dzp[s] > 0.f ? mul_(dzp[s], frcp(mul_(M.tp->lipschitz, inv_ld[s]))) : 0.f;
        x[s][0] = mul_(mul_(8.f, f[s]), inv_l);
        x[s][1] = mul_(mul_(8.f, dzp[s] > 0.f ? fpv[s] : f[s]), inv_l);
        x[s][2] = dzp[s] > 0.f ? mul_(8.f, dist) : 0.f;
        x[s][3] = mul_((float)(steps[s] + 1), 1.f / 64.f);
        x[s][4] = feat_prim;
        x[s][5] = feat_len;
        // a slot whose relaxation is off (after a rejected step) steps with
        // omega = 1 whatever the network says: no row for it
        live |= ((ray[s] >= 0 && !((relax_off >> s) & 1u)) ? 1u : 0u) << s;
      }
      __nv_bfloat16 *xs = reinterpret_cast<__nv_bfloat16 *>(wvals);
      mlp_omega_warp(LC.W, x, om, xs, wvals + 64 * 4, live);
    }
    int n_fin = 0;
#pragma unroll
    for (int s = 0; s < kR; ++s) {
      bool hit, exit;
      const bool was = ray[s] >= 0;
      step_slot(s, f[s], om[s], hit, exit);
      n_fin += __popc(__ballot_sync(0xFFFFFFFFu, was && (hit || exit || ray[s] < 0)));
      retire(s, hit, exit);
    }
    if (kShare && n_fin && lane == 0) atomicAdd(n_done, n_fin);
  }
  if (kCtaOk && cta != 0) {
    // After a CTA split every ray of its passes that hit is on the owner's
    // hit list: spread the list over the warps for refinement (warp w takes
    // the entries i = w mod kWarps; a ray's refinement does not depend on the
    // warp that runs it).
    const int warp_id = threadIdx.x >> 5;
    const int own = *(volatile int *)&cs->own, nh = *(volatile int *)&cs->nh;
    const uint16_t *oh = C.hits + (size_t)own * LC.L->max_tile_rays;
    const int mine = nh > warp_id ? (nh - warp_id + kWarps - 1) / kWarps : 0;
    if (cta == 2) {
      for (int j = lane; j < mine; j += 32) hits[n_hits + j] = oh[warp_id + kWarps * j];
      n_hits += mine;
      __syncwarp();
      cta_bar(1);
    } else {
      uint16_t keep[(kMaxTileRaysCta + 31) / 32];
#pragma unroll
      for (int q = 0; q < (kMaxTileRaysCta + 31) / 32; ++q) {
        const int j = lane + 32 * q;
        keep[q] = j < mine ? oh[warp_id + kWarps * j] : (uint16_t)0;
      }
      cta_bar(1);   // every helper has read its share
#pragma unroll
      for (int q = 0; q < (kMaxTileRaysCta + 31) / 32; ++q) {
        const int j = lane + 32 * q;
        if (j < mine) hits[j] = keep[q];
      }
      n_hits = mine;
      __syncwarp();
    }
  }
  c_rej += rejected;
  return live_steps;
}

// Hit refinement: Newton steps along the ray on f_A (value + derivative along
// d), then the gradient of f_A from three directional derivatives; a
// crossing that lies past z_end is handed to the next subfrustum.
template <int kFam>
__device__ __forceinline__ void finalize_hits(const MarchCtx &M, const CtaWork &C, const RecSrc &src, const SubInfo &inf,
                              const uint32_t *view, const uint16_t *hits, int n_hits, uint16_t *alive_out,
                              int *n_out, float2 *stk_lane, uint64_t &c_fin, unsigned long long *diag) {
  const int lane = threadIdx.x & 31;
  SmemStackD1 stk{stk_lane};
  const DevCamera &cam = *M.cam;
  for (int b = 0; b < n_hits; b += 32) {
    const int idx = b + lane;
    if (diag && lane == 0) {
      atomicAdd(&diag[3], 1ull);
      atomicAdd(&diag[4], (unsigned long long)min(32, n_hits - b));
    }
    const bool v = idx < n_hits;
    const int r = v ? hits[idx] : 0;
    float zz = v ? C.ray_z[r] : inf.z_begin;
    float d[3];
    pixel_ray(cam, M.x0 + r % M.tw, M.y0 + r / M.tw, d);
    const float dn = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const float lim = M.tp->newton_clamp / dn;
    // Newton on f_A along the ray; a ray stops at its own convergence
    // (|step| <= 1e-6 z, a few FP32 ulps of z), so its result does not
    // depend on the other rays of the warp.  Then the normal: gradient of f_A
    // from three axis derivatives at the final point (not reusing the last
    // Newton derivative: the field's gradient has kinks where the blend range
    // b_r reaches zero, and the previous Newton point may lie across one).
    // One evaluation call site serves both phases (instruction cache).
    bool beyond = false, done = !v;
    int n_eval = 0;
    float g[3] = {0.f, 0.f, 0.f};
    const int n_newton = M.tp->newton_iters;
#pragma unroll 1
    for (int it = 0; it < n_newton + 3; ++it) {
      const bool newton = it < n_newton;
      if (newton && !__any_sync(0xFFFFFFFFu, !done)) { it = n_newton - 1; continue; }
      const int k = it - n_newton;   // gradient axis (newton: < 0)
      Dual<1> pd[1][3], fd[1];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        pd[0][j].v = cam.o[j] + zz * d[j];
        pd[0][j].g[0] = newton ? d[j] : (j == k ? 1.f : 0.f);
      }
      eval_view_r<1, Dual<1>, SmemStackD1, kFam>(view, inf.n_view, src, pd, fd, stk);
      if (newton) {
        // a first sample inside the solid at the near plane: clipped hit
        if (it == 0 && zz <= kZNear && fd[0].v < -M.tp->eps) done = true;
        if (!done) {
          ++n_eval;
          beyond = false;
          if (fd[0].g[0] != 0.f && isfinite(fd[0].v)) {
            float step = -fd[0].v / fd[0].g[0];
            step = fminf(fmaxf(step, -lim), lim);
            beyond = zz + step > inf.z_end && fd[0].v > 0.f;
            const float zn = fminf(fmaxf(zz + step, inf.z_begin), inf.z_end);
            if (fabsf(zn - zz) <= 1e-6f * zz) done = true;
            zz = zn;
          } else {
            done = true;
          }
        }
      } else {
        g[0] = k == 0 ? fd[0].g[0] : g[0];
        g[1] = k == 1 ? fd[0].g[0] : g[1];
        g[2] = k == 2 ? fd[0].g[0] : g[2];
        ++n_eval;
      }
    }
    const bool back = v && beyond;
    if (back) {
      C.ray_z[r] = inf.z_end;
      C.ray_st[r] = C.ray_st[r] & 0xFFFFFFu;
    }
    append_rays(back, r, alive_out, n_out);
    if (v && !beyond) {
      const float gn = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
      const float ig = gn > 0.f ? 1.f / gn : 0.f;
      const size_t o = (size_t)(M.y0 + r / M.tw) * cam.W + (M.x0 + r % M.tw);
      M.out->depth[o] = zz * dn;
      M.out->normal[3 * o] = g[0] * ig;
      M.out->normal[3 * o + 1] = g[1] * ig;
      M.out->normal[3 * o + 2] = g[2] * ig;
      M.out->evals[o] = C.ray_st[r] & 0xFFFFFFu;
      M.out->flags[o] = 1;
      c_fin += (uint64_t)n_eval;
    }
  }
}

// ---- the tracing kernel ----------------------------------------------------------
// Three CTAs per SM: up to 170 registers per thread (the learned step's MLP
// fragments take it to 168) with ~57 KB of shared memory per CTA.
template <int INST>
__global__ void __launch_bounds__(kWarps * 32, (INST & kWideBit) ? 2 : 3)
k_trace(const Job *__restrict__ jobs, int n_jobs, TraceLaunch L) {
  constexpr int MODE = INST & ~(kFurtherBit | kStagedBit | kAllFamBit | kWideBit | kCtaBit);
  constexpr bool kCtaInst = (INST & kCtaBit) != 0;
  constexpr int kFam = (INST & kFurtherBit) ? ((INST & kAllFamBit) ? 2 : 1) : 0;
  constexpr bool kStaged = (INST & kStagedBit) != 0;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t s_item, s_rec;
  __shared__ int s_part;
  __shared__ SubInfo s_info[2];
  __shared__ int s_lvl_cur[kMaxLevels + 1];   // level cursors of the view build (warp 0)
  __shared__ ViewChunk s_vchunk;               // view build staging (warp 0)
  __shared__ int s_qhead[3], s_nctr[3];
  __shared__ int s_tqt[3], s_tqh[3], s_ndone[3], s_nidle[3];   // tail sharing per subfrustum slot
  __shared__ uint32_t s_steps;
  __shared__ unsigned long long s_dbg[8];
  __shared__ unsigned long long s_diag[7];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const CtaWork C = carve(smem, L, L.g_work ? L.g_work + (size_t)blockIdx.x * L.g_work_words : nullptr);
  float2 *stk_lane = C.stk + (size_t)warp * L.stack_slots * 32 + lane;
  float *wvals = reinterpret_cast<float *>(C.stk + (size_t)warp * L.stack_slots * 32);
  LearnCtx LC;
  LC.L = &L;
  LC.list_len = 0;
  LC.diag = L.tile_stats ? s_diag : nullptr;
  if (MODE == ST_STEP_LEARNED) LC.W = load_mlp(L.mlp, C.mlp);
  LC.stage = C.stage ? C.stage + (size_t)warp * kStageWords : nullptr;
  uint16_t *my_hits = C.hits + (size_t)warp * L.max_tile_rays;

  uint64_t c_steps = 0, c_prim = 0, c_op = 0, c_flops = 0, c_sub = 0, c_fin = 0, c_rej = 0, c_nev = 0, c_fev = 0;
  uint32_t c_err = 0;
  uint32_t g_sub = 0;   // subfrustums this CTA has started (tail-queue tag)
  // Shared memory is not cleared at launch: zero the tail queue so that no
  // stale entry can carry a tag of this launch (tags start at 1).
  for (int i = threadIdx.x; i < tq_cap(L); i += blockDim.x) C.tq[i] = 0ull;
  if (L.status && (*(volatile const uint32_t *)L.status & ST_STATUS_CAPACITY)) return;

  for (;;) {
    if (threadIdx.x == 0) {
      // ---- next work: the next whole tile; once all are handed out, a part
      // of a split tile ----
      uint32_t gt = 0xFFFFFFFFu, rec = 0;
      int part = 0;
      if (L.split && (L.heavy_len || L.heavy_thr)) gt = try_part(L, &rec, &part);
      if (gt == 0xFFFFFFFFu && *(volatile uint32_t *)L.item_counter < L.n_items) {
        if (L.split) {
          atomicAdd(&L.split[2], 1u);
          __threadfence();
        }
        const uint32_t it = atomicAdd(L.item_counter, 1u);
        if (it < L.n_items) gt = L.order ? L.order[it] : it;
        else if (L.split) atomicSub(&L.split[2], 1u);
      }
      if (gt == 0xFFFFFFFFu && L.split) gt = next_part(L, &rec, &part);
      s_item = gt;
      s_rec = rec;
      s_part = part;
    }
    __syncthreads();
    const uint32_t gtile = s_item;
    if (gtile == 0xFFFFFFFFu) break;
    const int part = s_part;
    const uint32_t *prec = part ? split_record(L, s_rec) : nullptr;
    bool split_done = false;   // this whole tile was split (its CTA keeps part 0) or cannot split
    const int jb = find_job_tile(jobs, n_jobs, gtile);
    const Job &job = jobs[jb];
    const DevScene &sc = job.sc;
    const uint32_t tile = gtile - job.tile_base;
    const int T = job.tl.tile;
    const int tx = (int)(tile % (uint32_t)job.tl.tiles_x), ty = (int)(tile / (uint32_t)job.tl.tiles_x);
    MarchCtx M;
    M.cam = &job.cam;
    M.tp = &job.tp;
    M.out = &job.out;
    M.x0 = tx * T;
    M.y0 = ty * T;
    M.tw = min(T, job.cam.W - M.x0);
    const int th = min(T, job.cam.H - M.y0);
    const int nr = M.tw * th;
    const uint32_t lbeg = job.tl.offsets[tile], len = job.tl.offsets[tile + 1] - lbeg;
    if (len > (uint32_t)L.act_cap) {
      // A list longer than the launch's active-set capacity (only possible
      // when a captured batch is replayed on edited scenes): report, no output.
      for (int r = threadIdx.x; r < nr; r += blockDim.x) write_miss(M, r, 0u, 0);
      c_err |= ST_STATUS_CAPACITY;
      if (L.split && !part && threadIdx.x == 0) atomicSub(&L.split[2], 1u);
      __syncthreads();
      continue;
    }
    // A heavy tile (long list) splits before its first subfrustum into about
    // one part per 512 entries (at most kHeavyParts): each part builds the
    // tile's views itself (no replay), and CTAs claim open parts before
    // whole tiles, so the tile's rays are traced by several CTAs from the
    // start instead of one CTA outlasting the frame.
    const uint32_t heavy_at = L.heavy_thr ? *L.heavy_thr : (L.heavy_len ? L.heavy_len : 0xFFFFFFFFu);
    const bool heavy = MODE != ST_STEP_RECORD && L.split && !part && len >= heavy_at && nr >= 2 * kSplitMinRays;
    if (L.split && !part && !heavy && (nr < 2 * kSplitMinRays || kSplitListBudget / max(len, 1u) < 2)) {
      // Too few rays or too long a list to split: release this tile's count
      // of whole tiles at once, so that CTAs out of work stop polling sooner.
      if (threadIdx.x == 0) atomicSub(&L.split[2], 1u);
      split_done = true;
    }
    LC.list_len = len;
    const float *zin_l = job.tl.z_in + lbeg;
    const float *zout_l = job.tl.z_out + lbeg;
    const uint32_t *prim_l = job.tl.prim + lbeg;
    const long long t_tile0 = clock64();
    long long t_prep = 0, t_march = 0, t_fin = 0;
    uint32_t s_sub = 0, s_maxview = 0;

    // K: the first subfrustum this CTA marches (a part of a split tile
    // resumes where the tile was split, after replaying its segmentation).
    int K = 0, n_pending = nr;
    if (!part) {
      for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        C.ray_z[r] = kZNear;
        C.ray_st[r] = 0u;
        pick(C.alive, 0)[r] = (uint16_t)r;
      }
    } else {
      // (defensive clamps: the record was written by this kernel)
      K = min((int)__ldcg(prec + 1), 2 * (int)len + 2);
      const int n = min((int)__ldcg(prec + 2), nr), P = max((int)__ldcg(prec + 3), 2);
      const uint32_t *ids = prec + 4;
      const float *rz = reinterpret_cast<const float *>(prec + 4 + L.max_tile_rays);
      const uint32_t *rst = prec + 4 + 2 * L.max_tile_rays;
      uint16_t *al = pick(C.alive, K & 1);
      for (int j = threadIdx.x; part + j * P < n; j += blockDim.x) {
        const int r = (int)__ldcg(ids + part + j * P);
        C.ray_z[r] = __ldcg(rz + r);
        C.ray_st[r] = __ldcg(rst + r);
        al[j] = (uint16_t)r;
      }
      n_pending = part < n ? (n - part + P - 1) / P : 0;
    }
    if (threadIdx.x == 0) {
      s_nctr[0] = 0; s_nctr[1] = 0; s_nctr[2] = 0;
      s_qhead[0] = 0; s_qhead[1] = 0; s_qhead[2] = 0;
      for (int i = 0; i < 3; ++i) { s_tqt[i] = 0; s_tqh[i] = 0; s_ndone[i] = 0; s_nidle[i] = 0; }
      if (kCtaInst) {
        // slot i is first used by subfrustum K + ((i - K) mod 3): its view buffer
        for (int i = 0; i < 3; ++i) s_ctash.sync[i] = CtaSync{0, 0, 0, 0, 0, 0, (K + (i - K % 3 + 3) % 3) & 1};
        s_ctash.info[0].n_top = 0;
        s_ctash.info[1].n_top = 0;
        s_ctash.cseg[0] = C.cseg[0];
        s_ctash.cseg[1] = C.cseg[1];
        s_ctash.ctop[0] = C.ctop[0];
        s_ctash.ctop[1] = C.ctop[1];
        s_ctash.crec = C.crec;
      }
      s_steps = 0u;
      for (int i = 0; i < 8; ++i) s_dbg[i] = 0ull;
      for (int i = 0; i < 7; ++i) s_diag[i] = 0ull;
    }
    // Split records (thread 0 reserves; all threads publish).  A record
    // resumes at subfrustum kn with the pending rays of alive[kn & 1]; part p
    // holds pending rays i = p (mod P); this CTA keeps part 0.
    auto reserve_split = [&](int P) -> int {
      if (P >= 2) {
        const uint32_t r = atomicAdd(&L.split[0], 1u);
        if (r < L.split_cap) s_rec = r; else P = 0;
      }
      return P >= 2 ? P : 0;
    };
    auto publish_split = [&](int kn, int P) {
      const uint32_t rr = s_rec;
      uint32_t *R = split_record(L, rr);
      uint16_t *al = pick(C.alive, kn & 1);   // the resume subfrustum's pending rays
      float *rz = reinterpret_cast<float *>(R + 4 + L.max_tile_rays);
      uint32_t *rst = R + 4 + 2 * L.max_tile_rays;
      for (int i = threadIdx.x; i < n_pending; i += blockDim.x) {
        const int r = al[i];
        R[4 + i] = (uint32_t)r;
        rz[r] = C.ray_z[r];
        rst[r] = C.ray_st[r];
      }
      if (threadIdx.x == 0) {
        R[0] = gtile;
        R[1] = (uint32_t)kn;
        R[2] = (uint32_t)n_pending;
        R[3] = (uint32_t)P;
      }
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        atomicExch(&L.split[4 + rr], (uint32_t)P);
        atomicSub(&L.split[2], 1u);
      }
      uint16_t *tmp = pick(C.alive, (kn + 1) & 1);   // free: written by subfrustum kn's march
      const int m = (n_pending + P - 1) / P;
      for (int j = threadIdx.x; j < m; j += blockDim.x) tmp[j] = al[j * P];
      __syncthreads();
      for (int j = threadIdx.x; j < m; j += blockDim.x) al[j] = tmp[j];
      __syncthreads();
      n_pending = m;
    };
    SegState sg;
    sg.next = 0; sg.n_act = 0; sg.cur = 0; sg.z_end = 0.f; sg.maxze = -INFINITY;
    int k = -1;
    // k < K only prepares subfrustum k + 1 (segmentation alone below K - 1);
    // one call site for the preparation keeps the kernel's code (and
    // instruction-fetch stalls) smaller.
    for (;; ++k) {
      const bool run = k >= K;
      SubInfo inf{};
      if (run) {
        inf = s_info[k & 1];
        if (inf.done || inf.err || n_pending == 0) {
          if (inf.err) c_err |= (uint32_t)inf.err;
          break;
        }
      }
      const int kk = run ? k : K;
      const int rd = kk % 3, wr = (kk + 1) % 3, rs = (kk + 2) % 3;
      const uint16_t *alive_in = pick(C.alive, kk & 1);
      uint16_t *alive_out = pick(C.alive, (kk + 1) & 1);
      if (run) {
        if (threadIdx.x == 0) {
          s_nctr[rs] = 0; s_qhead[rs] = 0; s_tqt[rs] = 0; s_tqh[rs] = 0; s_ndone[rs] = 0; s_nidle[rs] = 0;
          if (kCtaInst) s_ctash.sync[rs] = CtaSync{0, 0, 0, 0, 0, 0, k & 1};
        }
        ++g_sub;
      }
      if (warp == 0) {
        // The next subfrustum's view is built while the other warps march.
        const long long t0 = clock64();
        prepare_sub(sg, C, sc, job.tp, zin_l, zout_l, prim_l, len, (k + 1) & 1, L.stack_slots, L.dc_words,
                    &s_info[(k + 1) & 1], s_lvl_cur, &s_vchunk, L.tile_stats ? s_dbg : nullptr, k + 1 >= K,
                    kCtaInst ? L.cta_min_view : 0, L.view_cap, s_ctash.info, L.prune_views != 0);
        t_prep += clock64() - t0;
        if (run) {
          c_sub += 1;
          s_sub += 1;
          s_maxview = max(s_maxview, (uint32_t)inf.n_view);
        }
      }
      if (!run) {
        __syncthreads();
        if (heavy && k == -1) {
          if (threadIdx.x == 0) {
            const SubInfo nx = s_info[0];
            // about one part per 512 list entries (each part repeats the views)
            const int P = (!nx.done && !nx.err)
                              ? min(min(kHeavyParts, nr / kSplitMinRays), max(2, (int)(len / 512u)))
                              : 0;
            s_part = reserve_split(P);
          }
          __syncthreads();
          const int P = s_part;
          if (P >= 2) {
            publish_split(0, P);
            split_done = true;
          } else if (kSplitListBudget / max(len, 1u) < 2) {
            // not split (no record left): as a tile that cannot split
            if (threadIdx.x == 0) atomicSub(&L.split[2], 1u);
            split_done = true;
          }
        }
        continue;
      }
      if (inf.root_used) {
        const long long t0 = clock64();
        int n_hits = 0;
        const RecSrc src{sc.rec, pick(C.dc, k & 1)};
        const uint32_t ls = march_sub<MODE, kFam, kStaged, kCtaInst>(M, C, src, inf, pick(C.view, k & 1), pick(C.ops, k & 1), pick(C.lvl_off, k & 1), alive_in,
                                      n_pending, &s_qhead[rd], alive_out, &s_nctr[wr], my_hits, n_hits, stk_lane,
                                      wvals, 2 * L.stack_slots * 32, c_rej, LC, &s_tqt[rd], &s_tqh[rd], &s_ndone[rd],
                                      &s_nidle[rd], g_sub, c_err, rd);
        const long long t1 = clock64();
        c_steps += ls;
        c_prim += (uint64_t)ls * inf.n_prim;
        c_op += (uint64_t)ls * inf.n_op;
        c_flops += (uint64_t)ls * (inf.flops + kFlopsStep);
        c_nev += (uint64_t)ls * (uint32_t)inf.n_view;
        c_fev += (uint64_t)ls * (s_info[k & 1].flops_eval + kFlopsStep);
        finalize_hits<kFam>(M, C, src, inf, pick(C.view, k & 1), my_hits, n_hits, alive_out, &s_nctr[wr],
                                stk_lane, c_fin, LC.diag);
        if (L.tile_stats && lane == 0) {
          atomicAdd(&s_dbg[4], (unsigned long long)(clock64() - t1));
          atomicAdd(&s_dbg[7], (unsigned long long)(t1 - t0));
          if (warp == 0) {
            atomicAdd(&s_dbg[5], (unsigned long long)inf.n_view);
            atomicAdd(&s_dbg[6], (unsigned long long)inf.n_lvl);
          }
        }
        if (warp == 0) {
          t_march += t1 - t0;
          t_fin += clock64() - t1;
        }
        if (L.tile_stats) {
          uint32_t w = ls;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xFFFFFFFFu, w, o);
          if (lane == 0 && w) atomicAdd(&s_steps, w);
        }
      } else {
        // f_A = +inf in this subfrustum: no crossing, every pending ray moves on.
        for (int i = threadIdx.x; i < n_pending; i += blockDim.x) alive_out[i] = alive_in[i];
        if (threadIdx.x == 0) s_nctr[wr] = n_pending;
      }
      __syncthreads();
      n_pending = s_nctr[wr];
      if (MODE != ST_STEP_RECORD && L.split && !part && !split_done && n_pending >= 2 * kSplitMinRays) {
        // ---- a tile still tracing after L.split_cycles: publish parts 1..P-1
        // of its pending rays, keep part 0 ----
        if (threadIdx.x == 0) {
          int P = 0;
          const SubInfo nx = s_info[(k + 1) & 1];
          // Only once every tile has been handed out: before that, the other
          // CTAs have whole tiles to trace, and a split only adds the parts'
          // segmentation replays and view builds.
          if (!nx.done && !nx.err && clock64() - t_tile0 > L.split_cycles &&
              *(volatile uint32_t *)L.item_counter >= L.n_items) {
            // Each part repeats the tile's segmentation and view builds, whose
            // cost grows with the list: long lists split into fewer parts.
            P = min(min(kSplitMaxParts, n_pending / kSplitMinRays), (int)(kSplitListBudget / max(len, 1u)));
          }
          s_part = reserve_split(P);   // (s_part broadcasts P here; the tile's own part is in `part`)
        }
        __syncthreads();
        const int P = s_part;
        if (P >= 2) {
          publish_split(k + 1, P);
          split_done = true;
        }
      }
    }
    if (L.split && !part && !split_done && threadIdx.x == 0) atomicSub(&L.split[2], 1u);
    // ---- rays still pending when the list is exhausted: misses ----
    for (int i = threadIdx.x; i < n_pending; i += blockDim.x) {
      const int r = pick(C.alive, k & 1)[i];
      write_miss(M, r, C.ray_st[r] & 0xFFFFFFu, 0);
    }
    __syncthreads();
    if (L.tile_stats && threadIdx.x == 0 && !part) {
      uint32_t *ts = L.tile_stats + (size_t)gtile * kTileStatWords;
      for (int i = 0; i < 7; ++i) ts[16 + i] = (uint32_t)min(s_diag[i], 0xFFFFFFFFull);
      ts[8] = (uint32_t)(s_dbg[0] >> 4);
      ts[9] = (uint32_t)(s_dbg[1] >> 4);
      ts[10] = (uint32_t)(s_dbg[2] >> 4);
      ts[11] = (uint32_t)(s_dbg[3] >> 4);
      ts[12] = (uint32_t)(s_dbg[4] >> 4);
      ts[13] = (uint32_t)s_dbg[5];
      ts[14] = (uint32_t)s_dbg[6];
      ts[15] = (uint32_t)(s_dbg[7] >> 4);
      ts[0] = (uint32_t)((clock64() - t_tile0) >> 4);
      ts[1] = (uint32_t)(t_prep >> 4);
      ts[2] = (uint32_t)(t_march >> 4);
      ts[3] = (uint32_t)(t_fin >> 4);
      ts[4] = s_sub;
      ts[5] = s_steps;
      ts[6] = s_maxview;
      ts[7] = len;
    }
    __syncthreads();
  }

  if (L.status && c_err && lane == 0) atomicOr(L.status, c_err);
  if (L.counters) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      c_steps += __shfl_xor_sync(0xFFFFFFFFu, c_steps, o);
      c_prim += __shfl_xor_sync(0xFFFFFFFFu, c_prim, o);
      c_op += __shfl_xor_sync(0xFFFFFFFFu, c_op, o);
      c_flops += __shfl_xor_sync(0xFFFFFFFFu, c_flops, o);
      c_nev += __shfl_xor_sync(0xFFFFFFFFu, c_nev, o);
      c_fev += __shfl_xor_sync(0xFFFFFFFFu, c_fev, o);
      c_fin += __shfl_xor_sync(0xFFFFFFFFu, c_fin, o);
      c_rej += __shfl_xor_sync(0xFFFFFFFFu, c_rej, o);
    }
    if (lane == 0) {
      atomicAdd((unsigned long long *)&L.counters[5], (unsigned long long)c_rej);
      atomicAdd((unsigned long long *)&L.counters[0], (unsigned long long)c_steps);
      atomicAdd((unsigned long long *)&L.counters[1], (unsigned long long)c_prim);
      atomicAdd((unsigned long long *)&L.counters[2], (unsigned long long)c_op);
      atomicAdd((unsigned long long *)&L.counters[3], (unsigned long long)c_flops);
      if (warp == 0) atomicAdd((unsigned long long *)&L.counters[4], (unsigned long long)c_sub);
      atomicAdd((unsigned long long *)&L.counters[6], (unsigned long long)c_fin);
      if (c_err) atomicOr((unsigned long long *)&L.counters[7], (unsigned long long)c_err);
      atomicAdd((unsigned long long *)&L.counters[8], (unsigned long long)c_nev);
      atomicAdd((unsigned long long *)&L.counters[9], (unsigned long long)c_fev);
    }
  }
}

// ---- work order: longest tile lists first ----------------------------------------
// One CTA: histogram of list lengths (4096 bins, longer lists share the
// last), bins scanned from the longest down, tiles scattered.  Heavy tiles
// then start while every SM is free instead of finishing last.
__global__ void __launch_bounds__(1024) k_tile_order(const Job *jobs, int n_jobs, uint32_t n_tiles, uint32_t *order,
                                                     uint32_t heavy_rank, uint32_t heavy_min, uint32_t *heavy_thr) {
  constexpr int kBins = 4096;
  __shared__ uint32_t cnt[kBins];
  __shared__ uint32_t s_warp[32];
  auto tile_bin = [&](uint32_t g) -> uint32_t {
    const Job &job = jobs[find_job_tile(jobs, n_jobs, g)];
    const uint32_t t = g - job.tile_base;
    return min(job.tl.offsets[t + 1] - job.tl.offsets[t], (uint32_t)kBins - 1u);
  };
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) cnt[i] = 0u;
  __syncthreads();
  for (uint32_t g = threadIdx.x; g < n_tiles; g += blockDim.x) atomicAdd(&cnt[tile_bin(g)], 1u);
  __syncthreads();
  // exclusive scan over bins in descending order: thread t owns 4 bins
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t v[4], sum = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    v[q] = cnt[kBins - 1 - (threadIdx.x * 4 + q)];
    sum += v[q];
  }
  uint32_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = s_warp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  uint32_t base = (warp > 0 ? s_warp[warp - 1] : 0u) + x - sum;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    cnt[kBins - 1 - (threadIdx.x * 4 + q)] = base;   // start of the bin in the order
    base += v[q];
  }
  __syncthreads();
  for (uint32_t g = threadIdx.x; g < n_tiles; g += blockDim.x) order[atomicAdd(&cnt[tile_bin(g)], 1u)] = g;
  if (heavy_thr) {
    // Early-split threshold: the list length of the heavy_rank-th longest
    // tile, at least heavy_min (lists of 4095+ entries share the top bin, in
    // any order; ties are all heavy).
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t thr = 0xFFFFFFFFu;
      if (heavy_rank > 0 && n_tiles > 0) {
        const uint32_t g = order[min(heavy_rank, n_tiles) - 1];
        const Job &job = jobs[find_job_tile(jobs, n_jobs, g)];
        const uint32_t t = g - job.tile_base;
        thr = max(job.tl.offsets[t + 1] - job.tl.offsets[t], heavy_min);
      }
      *heavy_thr = thr;
    }
  }
}

void launch_tile_order(const Job *jobs, int n_jobs, uint32_t n_tiles, uint32_t *order, cudaStream_t s,
                       uint32_t heavy_rank, uint32_t heavy_min, uint32_t *heavy_thr) {
  if (n_tiles)
    count_launch(), k_tile_order<<<1, 1024, 0, s>>>(jobs, n_jobs, n_tiles, order, heavy_rank, heavy_min, heavy_thr);
  else if (heavy_thr)
    cudaMemsetAsync(heavy_thr, 0xFF, sizeof(uint32_t), s);
}

// ---- inspection kernels: the same view build and evaluator as k_trace ----------
// method 0: the tracer's warp-parallel builder (build_view_lca); method 1:
// Algorithm 1 as stated (one lane, fast ancestor pointers); method 2: method
// 0 without the subtrees the usage rewrite discards (compact_live_view), the
// view st_trace evaluates by default.  One warp;
// `scratch` holds the builder's work arrays (pruned_view_scratch_words).
__global__ void k_pruned_view(DevScene sc, const uint32_t *act, int n, uint32_t *view, uint32_t *vaddr,
                              int32_t *info, uint32_t *scratch, int stack_cap, int method) {
  if (blockIdx.x != 0) return;
  ViewInfo vi;
  int n_lvl = 0;
  if (method != 1) {
    __shared__ ViewChunk vch;
    uint32_t *stk = scratch;   // 16-byte aligned (device allocation base)
    uint2 *ops = reinterpret_cast<uint2 *>(scratch + align16((size_t)6 * (stack_cap + 2) * 4) / 4);
    uint2 *sort_tmp = ops + n;
    int *lvl_off = reinterpret_cast<int *>(sort_tmp + n);
    int *lvl_cur = lvl_off + kMaxLevels + 1;
    vi = vaddr ? build_view_lca<true>(sc, act, n, view, vch, ops, sort_tmp, lvl_off, lvl_cur, stk, stack_cap, vaddr, &n_lvl)
               : build_view_lca<false>(sc, act, n, view, vch, ops, sort_tmp, lvl_off, lvl_cur, stk, stack_cap, vaddr, &n_lvl);
    if (method == 2 && !vi.err && vi.root_used && n_lvl > 0) {
      int nop2 = 0, nlvl2 = 0;
      uint32_t fl2 = 0;
      const int n2 = compact_live_view(view, vi.n_view, ops, lvl_off, lvl_cur, n_lvl, sort_tmp, &nop2, &nlvl2, &fl2,
                                       vaddr);
      if (n2 > 0) vi.n_view = n2;
    }
  } else {
    if (threadIdx.x != 0) return;
    vi = build_view(sc, act, n, view, scratch, stack_cap, vaddr);
  }
  if (threadIdx.x == 0) {
    info[0] = vi.n_view;
    info[1] = vi.root_used;
    info[2] = vi.err;
    info[3] = vi.n_prim;
  }
}

size_t pruned_view_scratch_words(int n, int stack_cap) {
  return align16((size_t)6 * (stack_cap + 2) * 4) / 4 + (size_t)n * 4 + 2 * (kMaxLevels + 1) + 16;
}

// f_A (and optionally its forward-mode gradient) at arbitrary points for a
// view already built by k_pruned_view; one thread per point.
__global__ void k_eval_view(DevScene sc, const uint32_t *view, const int32_t *info, const float *pts, int npts,
                            float *f, float *grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npts) return;
  const int n_view = info[0];
  if (info[2] != 0 || !info[1]) {
    f[i] = INFINITY;
    if (grad) { grad[3 * i] = 0.f; grad[3 * i + 1] = 0.f; grad[3 * i + 2] = 0.f; }
    return;
  }
  if (!grad) {
    const float p[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
    LocalStack<float> ls;
    f[i] = eval_view<float>(view, n_view, RecSrc{sc.rec, nullptr}, p, ls);
  } else {
    Dual<3> p[3];
    for (int k = 0; k < 3; ++k) {
      p[k].v = pts[3 * i + k];
      p[k].g[0] = k == 0; p[k].g[1] = k == 1; p[k].g[2] = k == 2;
    }
    LocalStack<Dual<3>> ls;
    Dual<3> r = eval_view<Dual<3>>(view, n_view, RecSrc{sc.rec, nullptr}, p, ls);
    f[i] = r.v;
    grad[3 * i] = r.g[0]; grad[3 * i + 1] = r.g[1]; grad[3 * i + 2] = r.g[2];
  }
}

// The tracer's view build followed by the warp-wide level evaluation of the
// tail mode, one point after another (one warp).  info: view length, root
// usage bit, error, operator levels of the schedule (0: no schedule; f is
// then NaN).  `scratch` as for k_pruned_view plus 2n floats of node values.
__global__ void k_eval_levels(DevScene sc, const uint32_t *act, int n, uint32_t *view, int32_t *info,
                              uint32_t *scratch, int stack_cap, const float *pts, int npts, float *f) {
  if (blockIdx.x != 0) return;
  __shared__ ViewChunk vch;
  uint32_t *stk = scratch;
  uint2 *ops = reinterpret_cast<uint2 *>(scratch + align16((size_t)6 * (stack_cap + 2) * 4) / 4);
  uint2 *sort_tmp = ops + n;
  int *lvl_off = reinterpret_cast<int *>(sort_tmp + n);
  int *lvl_cur = lvl_off + kMaxLevels + 1;
  float *vals = reinterpret_cast<float *>(lvl_cur + kMaxLevels + 1);
  int n_lvl = 0;
  const ViewInfo vi = build_view_lca<false>(sc, act, n, view, vch, ops, sort_tmp, lvl_off, lvl_cur, stk, stack_cap,
                                            nullptr, &n_lvl);
  const bool ok = !vi.err && vi.root_used && n_lvl > 0;
  if (threadIdx.x == 0) {
    info[0] = vi.n_view;
    info[1] = vi.root_used;
    info[2] = vi.err;
    info[3] = ok ? n_lvl : 0;
  }
  __syncwarp();
  const RecSrc src{sc.rec, nullptr};
  for (int i = 0; i < npts; ++i) {
    float v = NAN;
    if (ok) {
      const float p[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
      v = tail_eval<2>(view, vi.n_view, ops, lvl_off, n_lvl, src, p, vals);
    }
    if (threadIdx.x == 0) f[i] = v;
  }
}

size_t eval_levels_scratch_words(int n, int stack_cap) { return pruned_view_scratch_words(n, stack_cap) + 2 * (size_t)n; }

void launch_eval_levels(const DevScene &sc, const uint32_t *act, int n, uint32_t *view, int32_t *info,
                        uint32_t *scratch, int stack_cap, const float *pts, int npts, float *f, cudaStream_t s) {
  count_launch(), k_eval_levels<<<1, 32, 0, s>>>(sc, act, n, view, info, scratch, stack_cap, pts, npts, f);
}

void launch_pruned_view(const DevScene &sc, const uint32_t *act, int n, uint32_t *view, uint32_t *vaddr,
                        int32_t *info, uint32_t *scratch, int stack_cap, int method, cudaStream_t s) {
  count_launch(), k_pruned_view<<<1, 32, 0, s>>>(sc, act, n, view, vaddr, info, scratch, stack_cap, method);
}

void launch_eval_view(const DevScene &sc, const uint32_t *view, const int32_t *info, const float *pts, int npts,
                      float *f, float *grad, cudaStream_t s) {
  if (npts > 0) count_launch(), k_eval_view<<<(npts + 127) / 128, 128, 0, s>>>(sc, view, info, pts, npts, f, grad);
}

// Kernel instances: every step mode, with or without the out-of-line
// primitive families (torus, sphere-cone, ellipsoid, rounded triangle,
// bounded quadric).  Scenes of spheres, rounded boxes and capsules run the
// lean instance: its interpreter has no call to the further families, whose
// registers otherwise count for the whole kernel (measured on B300: 1080p
// trace 4-5 % faster).
template <class F>
static auto with_instance(const TraceLaunch &L, F &&f) {
#define ST_INST1(M)                                                                    \
  return L.further == 2 ? f(std::integral_constant<int, (M) | kFurtherBit | kAllFamBit>{}) \
         : L.further    ? f(std::integral_constant<int, (M) | kFurtherBit>{})               \
                        : f(std::integral_constant<int, (M)>{})
#define ST_INST(M)                                                                \
  if (!L.staged) { ST_INST1(M); }                                                \
  if constexpr ((M) != ST_STEP_RECORD) {                                         \
    if (L.cta_min_view > 0) {                                                    \
      if (L.dc_words > 640) { ST_INST1((M) | kStagedBit | kCtaBit | kWideBit); } \
      ST_INST1((M) | kStagedBit | kCtaBit);                                      \
    }                                                                            \
  }                                                                              \
  ST_INST1((M) | kStagedBit)
  switch (L.step_mode) {
    case ST_STEP_OVERRELAX: ST_INST(ST_STEP_OVERRELAX);
    case ST_STEP_CROSSING: ST_INST(ST_STEP_CROSSING);
    case ST_STEP_LEARNED: ST_INST(ST_STEP_LEARNED);
    case ST_STEP_RECORD: ST_INST(ST_STEP_RECORD);
    default: ST_INST(ST_STEP_PLAIN);
  }
#undef ST_INST
#undef ST_INST1
}

template <int MODE>
static cudaError_t trace_config(const TraceLaunch &L, int n_sm, int *grid, size_t *smem) {
  *smem = smem_per_cta(L);
  cudaError_t e = cudaFuncSetAttribute(k_trace<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace<MODE>, kWarps * 32, *smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *grid = n_sm * per_sm;
  return cudaSuccess;
}

cudaError_t trace_plan(const TraceLaunch &L, int n_sm, int *grid, size_t *smem) {
  return with_instance(L, [&](auto m) { return trace_config<decltype(m)::value>(L, n_sm, grid, smem); });
}

cudaError_t trace_launch_planned(const Job *jobs, int n_jobs, const TraceLaunch &L, int grid, size_t smem,
                                 cudaStream_t s) {
  return with_instance(L, [&](auto m) {
    count_launch(), k_trace<decltype(m)::value><<<grid, kWarps * 32, smem, s>>>(jobs, n_jobs, L);
    return cudaGetLastError();
  });
}

cudaError_t trace_launch(const Job *jobs, int n_jobs, const TraceLaunch &L, int n_sm, cudaStream_t s) {
  int grid = 0;
  size_t smem = 0;
  cudaError_t e = trace_plan(L, n_sm, &grid, &smem);
  if (e != cudaSuccess) return e;
  return trace_launch_planned(jobs, n_jobs, L, grid, smem, s);
}

int trace_ctas_per_sm(const TraceLaunch &L) {
  int grid = 0;
  size_t smem = 0;
  if (trace_plan(L, 1, &grid, &smem) != cudaSuccess) return 0;
  return grid;
}

}  // namespace st
