// st_kernels.h -- launch wrappers shared between the C ABI and the kernels.
#pragma once
#include <cstdint>

#include "st_internal.h"

namespace st {

struct Pair {          // a surviving (primitive, tile) pair of the culling pass
  uint32_t tile, rank;
  float z_in, z_out;
  uint32_t addr;
};

constexpr uint32_t kSortSmall = 4096;    // shared-memory sort, 48 KB
constexpr uint32_t kSortLarge = 16384;   // shared-memory sort, 192 KB

void scan_u32(const uint32_t *in, uint32_t *out, uint32_t n, uint32_t *block_sums, uint32_t *total,
              uint32_t *max_out, uint32_t *tail, cudaStream_t s);
uint32_t scan_block_count(uint32_t n);

void launch_prim_bounds(const Job *jobs, int n_jobs, uint32_t n_prims, uint32_t *cand_count, int4 *rects,
                        cudaStream_t s);
void launch_cull_pairs(const Job *jobs, int n_jobs, const uint32_t *cand_off, uint32_t n_prims,
                       const uint32_t *cand_total, const int4 *rects, uint32_t *tile_count, Pair *pairs,
                       uint32_t pair_cap, uint32_t *pair_counter, int n_sm, cudaStream_t s,
                       bool stri);   // stri: some scene holds rounded triangles (second launch)
void launch_scatter_sort(const Pair *pairs, const uint32_t *pair_counter, uint32_t pair_cap,
                         const uint32_t *offsets, uint32_t n_tiles, uint32_t max_overlap, uint64_t *keys,
                         float *z_out_tmp, float *z_in, float *z_out, uint32_t *prim, int n_sm, cudaStream_t s,
                         const uint32_t *abort = nullptr, uint32_t *long_list = nullptr,
                         uint32_t *long_count = nullptr);
// Lists longer than kSortLarge (launch_scatter_sort calls it when it is given
// a tile-sized list buffer and a counter): sorted chunks, then merge passes.
void launch_long_sort(const uint32_t *offsets, uint32_t n_tiles, uint32_t max_len, uint64_t *keys,
                      float *z_out_tmp, float *z_in, float *z_out, uint32_t *prim, uint32_t *list,
                      uint32_t *count, int n_sm, cudaStream_t s, const uint32_t *abort = nullptr);
void launch_check_capacity(const uint32_t *pair_counter, uint32_t pair_cap, const uint32_t *max_overlap,
                           uint32_t overlap_cap, uint32_t *status, cudaStream_t s);
cudaError_t cull_set_attributes();
// Sort of CSR segments by (z_in, address) keys: copy of 1-entry segments, and
// shared-memory sorts of segments with min_len < length <= max_len.
void launch_copy_short(const uint32_t *offsets, uint32_t n_segs, const uint64_t *keys, const float *z_out_tmp,
                       float *z_in, float *z_out, uint32_t *prim, cudaStream_t s, const uint32_t *abort = nullptr);
void launch_tile_sort_range(const uint32_t *offsets, uint32_t n_segs, uint32_t max_len, uint32_t min_len,
                            const uint64_t *keys, const float *z_out_tmp, float *z_in, float *z_out,
                            uint32_t *prim, int n_sm, cudaStream_t s, const uint32_t *abort = nullptr);

// ---- non-synchronized per-pixel variants (st_dexel.cu) ----
struct DexelLaunch {
  const uint32_t *offsets;   // [W * H + 1] per-pixel CSR of the dexel buffer
  const float *z_in, *z_out;
  const uint32_t *prim;
  uint2 *act;                // per-thread active sets: entry i of thread t at
                             // act[i * n_threads + t] (address, z_out bits)
  uint32_t n_threads;        // grid threads (stride of act)
  uint32_t *pixel_counter;   // zeroed before the launch
  uint64_t *counters;        // optional ST_NUM_COUNTERS
};
// Count (fill = false) or write (fill = true) the per-pixel fragments of the
// tile lists in job.tl; pix_off: exclusive scan of the counts.
void launch_dexel_pass(const Job &job, bool fill, uint32_t *count, const uint32_t *pix_off, uint64_t *keys,
                       float *zo_tmp, cudaStream_t s);
void launch_segment_sort(const uint32_t *offsets, uint32_t n_segs, uint32_t max_len, const uint64_t *keys,
                         const float *z_out_tmp, float *z_in, float *z_out, uint32_t *prim, int n_sm,
                         cudaStream_t s);
cudaError_t launch_eval_sparse(const DevScene &sc, const uint32_t *act, int n, const float *pts, int npts,
                               int fast, float *f, uint32_t *status, cudaStream_t s);
cudaError_t dexel_trace_grid(int fast, int n_sm, int *grid);
cudaError_t launch_trace_dexel(const Job &job, const DexelLaunch &D, int fast, int grid, cudaStream_t s);

// Status word bits of batched launches (device, OR-accumulated).
constexpr uint32_t ST_STATUS_VIEW = 1u;       // a pruned view exceeded its capacity
constexpr uint32_t ST_STATUS_STACK = 2u;      // evaluation stack overflow
constexpr uint32_t ST_STATUS_CAPACITY = 4u;   // entries / list length beyond the planned buffers
constexpr uint32_t ST_STATUS_WAIT = 8u;       // a bounded wait inside a CTA expired

// Tracing launch: shared memory per CTA, and the per-CTA work areas (active
// sets, views, level schedules) in shared or global memory; see st_trace.cu.
struct TraceLaunch {
  int32_t max_tile_rays;   // tile * tile of the largest tile in the launch
  int32_t act_cap;         // active-set capacity (>= longest tile list)
  int32_t view_cap;        // 2 * act_cap - 1
  int32_t stack_slots;     // evaluation stack slots per lane
  int32_t work_in_smem;    // 1: active set + view in shared memory
  int32_t staged;          // 1: views evaluated in staged chunks (trace_staged)
  int32_t dc_words;        // shared parameter cache per view buffer (float4 words)
  uint32_t *g_work;        // global per-CTA work areas (when not in shared
                           // memory), one per CTA of the persistent grid,
                           // indexed by blockIdx.x
  uint32_t g_work_words;   // words per CTA in g_work
  uint32_t n_items;        // total (job, tile) work items
  uint32_t *item_counter;  // zeroed before launch
  uint64_t *counters;      // optional ST_NUM_COUNTERS
  uint32_t *tile_stats;    // optional [n_items][16] diagnostics
  int32_t step_mode;       // selects the kernel instantiation
  const void *mlp;         // packed MLP weights (learned step)
  float *records;          // recording mode: [rec_cap][8] step records
  uint32_t rec_cap;
  uint32_t *rec_count;     // device counter (zeroed by the caller)
  int32_t rec_stride;      // record rays whose pixel index % stride == 0
  uint32_t *status;        // optional status word (ST_STATUS_*); the kernel
                           // returns at once when the capacity bit is set
  const uint32_t *order;   // optional [n_items] global tile per work item
                           // (launch_tile_order: longest list first)
  uint32_t *split;         // optional split area (tiles split across CTAs,
                           // see st_trace.cu); its first 4 + 2 split_cap
                           // words are zeroed before the launch
  uint32_t split_cap;      // split records in the area
  long long split_cycles;  // a tile still tracing after this many SM cycles
                           // splits at its next subfrustum boundary
  uint32_t heavy_len;      // a tile whose list holds at least this many
                           // entries splits before its first subfrustum,
                           // and CTAs claim open parts before whole tiles
                           // (0: no early splits)
  uint32_t idle_spins;     // polls of a warp waiting for rays of its tile
                           // (0: built-in bound)
  uint32_t split_spins;    // polls of a CTA waiting for split parts
                           // (0: built-in bound)
  int32_t further;         // kernel instance by the scenes' primitive families:
                           // 0 spheres, rounded boxes and capsules only; 1 also
                           // tori, sphere-cones, ellipsoids; 2 any family
  const uint32_t *heavy_thr;  // optional device word: early-split threshold
                              // (written by launch_tile_order); overrides
                              // heavy_len
  int32_t prune_views;     // 1: views without the subtrees their usage
                           // rewrite discards (see live_prims)
  int32_t cta_min_view;    // staged launches: views of at least this many
                           // nodes are prepared for the CTA-split evaluation
                           // of a subfrustum's last rays (0: never; the work
                           // areas then hold no split arrays)
};

// Split area sizing: words per record (header, pending ray ids, depth and
// steps by ray id), records of a launch (at most one per tile, about 16 MiB
// in all), total words and the words to zero before each launch.
__host__ __device__ inline size_t split_rec_words(int max_tile_rays) { return 4 + 3 * (size_t)max_tile_rays; }
inline uint32_t trace_split_cap(int max_tile_rays, uint32_t n_items) {
  const size_t by_size = (size_t(16) << 20) / (4 * split_rec_words(max_tile_rays));
  return (uint32_t)(n_items < by_size ? n_items : by_size);
}
inline size_t trace_split_words(int max_tile_rays, uint32_t cap) {
  return 4 + 2 * (size_t)cap + (size_t)cap * split_rec_words(max_tile_rays);
}
inline size_t trace_split_zero_bytes(uint32_t cap) { return 4 * (4 + 2 * (size_t)cap); }
// st_trace_opts::split_kcycles -> SM cycles (-1: tiles never split).
inline long long trace_split_cycles(int32_t split_kcycles) {
  if (split_kcycles < 0) return -1;
  return 1000ll * (split_kcycles > 0 ? split_kcycles : 2000);
}

// st_trace_opts::heavy_split_len -> TraceLaunch::heavy_len (0: off).
// Early splits are off by default: each part of a split tile repeats the
// tile's view builds, and on the 10k clustered scene, where hundreds of tiles
// hold 2,000-4,000 entries and view preparation is most of a tile's time,
// splitting the longest lists early was slower (measured on B300 at
// 1920x1080: learned trace 109 ms without, 191-194 ms with thresholds
// 1500-3000; at 960x540 132 vs 135-143 ms; at 3840x2160 145 vs 325 ms).
// Views evaluated in staged chunks (shared-memory stages filled by
// asynchronous copies): launches whose views live in global memory and can
// outgrow the shared parameter cache.  Short views stay on the plain
// interpreter, for which the view words' loads hit L1 (measured on B300:
// staging costs 4-12 % on 1,024 primitives at 1920x1080 and saves ~20 % on
// 10k clustered primitives).
inline int32_t trace_staged(const TraceLaunch &L) { return !L.work_in_smem && L.view_cap > 2048 ? 1 : 0; }
// st_trace_opts::cta_eval_min_view -> TraceLaunch::cta_min_view (staged
// launches only; 0 takes the default: on for st_trace launches with the
// large parameter cache, i.e. bound by their heaviest tiles, off otherwise.
// Measured on B300 with views without discarded subtrees: 10k clustered
// primitives at 1920x1080 (large cache) 4-10 % faster with it, at 3840x2160
// (small cache) 2-4 % slower, the 64-scene batch 24 % slower.
constexpr int32_t kCtaMinViewDefault = 1024;
inline int32_t trace_cta_min_view(const TraceLaunch &L, int32_t opt, bool on_by_default) {
  if (!L.staged || opt < 0 || (opt == 0 && !(on_by_default && L.dc_words > 640))) return 0;
  return opt > 0 ? (opt < 64 ? 64 : opt) : kCtaMinViewDefault;
}
inline uint32_t trace_heavy_len(int32_t opt) { return opt > 0 ? (uint32_t)opt : 0u; }
// st_trace_opts::heavy_split_rank -> rank of the list-length threshold taken
// on the device (0: no rank rule), and the least list length it splits.
constexpr int32_t kHeavyRankDefault = 0;
inline uint32_t trace_heavy_rank(int32_t len_opt, int32_t rank_opt) {
  if (len_opt > 0 || rank_opt < 0) return 0u;
  return (uint32_t)(rank_opt > 0 ? rank_opt : kHeavyRankDefault);
}
inline uint32_t trace_heavy_min(uint64_t n_entries, uint32_t n_tiles) {
  const double m = n_tiles ? 4.0 * (double)n_entries / (double)n_tiles : 0.0;
  return (uint32_t)(m > 1024.0 ? (m < 4.0e9 ? m : 4.0e9) : 1024.0);
}

constexpr int ST_STEP_RECORD = 15;  // plain stepping that records training data (internal)

size_t trace_smem_per_warp(const TraceLaunch &L);
uint32_t trace_work_words(const TraceLaunch &L);
// Parameter cache words per view buffer for a launch whose views hold up to
// view_cap nodes, whose longest tile list has max_overlap entries out of
// n_entries in all, on n_sm SMs.
int trace_dcache_words(int view_cap, uint32_t max_overlap, uint64_t n_entries, int n_sm);
cudaError_t trace_launch(const Job *jobs, int n_jobs, const TraceLaunch &L, int n_sm, cudaStream_t s);
// Split form for graph capture: trace_plan sets the kernel attributes and
// returns the persistent grid and shared memory size (call before capture);
// trace_launch_planned only enqueues the launch.
cudaError_t trace_plan(const TraceLaunch &L, int n_sm, int *grid, size_t *smem);
cudaError_t trace_launch_planned(const Job *jobs, int n_jobs, const TraceLaunch &L, int grid, size_t smem,
                                 cudaStream_t s);
int trace_warps_per_cta();
// Work order of a trace launch: the jobs' n_tiles global tiles sorted by
// A-buffer list length, longest first (counting sort; equal lengths in any
// order -- results do not depend on the order tiles are traced in).
// heavy_thr (optional): receives the early-split threshold, the list length
// of the heavy_rank-th longest tile but at least heavy_min (0xFFFFFFFF when
// heavy_rank is 0).
void launch_tile_order(const Job *jobs, int n_jobs, uint32_t n_tiles, uint32_t *order, cudaStream_t s,
                       uint32_t heavy_rank = 0, uint32_t heavy_min = 0, uint32_t *heavy_thr = nullptr);
int trace_ctas_per_sm(const TraceLaunch &L);
void launch_pruned_view(const DevScene &sc, const uint32_t *act, int n, uint32_t *view, uint32_t *vaddr,
                        int32_t *info, uint32_t *scratch, int stack_cap, int method, cudaStream_t s);
size_t pruned_view_scratch_words(int n, int stack_cap);
size_t eval_levels_scratch_words(int n, int stack_cap);
void launch_eval_levels(const DevScene &sc, const uint32_t *act, int n, uint32_t *view, int32_t *info,
                        uint32_t *scratch, int stack_cap, const float *pts, int npts, float *f, cudaStream_t s);
void launch_eval_view(const DevScene &sc, const uint32_t *view, const int32_t *info, const float *pts, int npts,
                      float *f, float *grad, cudaStream_t s);

}  // namespace st
