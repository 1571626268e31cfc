// st_noalloc.cu -- st_trace_noalloc: the tracing call without any device
// allocation.  Its scratch memory lives in one file-scope device array of
// fixed size that every device loading the library keeps until the process
// exits.  Layout (byte offsets): [0] work-queue counter, [4] status word,
// [8] early-split threshold, [256] the job record, then the tile order (one word per tile), then for
// long tile lists the per-CTA work areas, then as many records of tiles split
// across CTAs as fit.
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>

#include "st_kernels.h"

namespace st {
void scene_facts(const st_scene *s, DevScene *sc, int *stack_depth, double *diameter, double *extent, int *n_sm);
TraceParams make_trace_params(const st_trace_opts &o, double diameter, double extent);
int trace_status_code(const uint32_t *status, cudaStream_t st, const char *who);
int scene_further_level(const st_scene *s);
}

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr size_t kCounterOff = 0;                     // uint32 work-queue counter
constexpr size_t kStatusOff = 4;                      // uint32 device status word
constexpr size_t kHeavyOff = 8;                       // uint32 early-split threshold
constexpr size_t kJobOff = 256;                       // st::Job record
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_trace_scratch[kScratchBytes];

std::mutex g_scratch_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};
// Layout of the last call (st_trace_noalloc_last_layout): work areas in the
// scratch array, scratch bytes in use, split records.
std::atomic<uint64_t> g_last_work_in_scratch{0}, g_last_used{0}, g_last_split_cap{0};

// The host-side name of g_trace_scratch is not a device address: resolve it
// once per device, with that device current.
int scratch_for_current_device(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    st::set_error(std::string("st_trace_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return ST_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    st::set_error("st_trace_noalloc: device ordinal out of range");
    return ST_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_trace_scratch);
    if (e != cudaSuccess || !ptr) {
      st::set_error(std::string("st_trace_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return ST_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<unsigned char *>(ptr);
  }
  *out = g_scratch_addr[dev];
  return ST_OK;
}

// Writes the job record into the scratch array from the launch parameters
// (no host staging buffer).
__global__ void k_put_job(st::Job job, st::Job *dst) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dst = job;
}

}  // namespace

#define NA_CK(call)                                                         \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) {                                                \
      st::set_error(std::string("st_trace_noalloc: " #call ": ") + cudaGetErrorString(e_)); \
      return ST_ERR_CUDA;                                                   \
    }                                                                       \
  } while (0)

extern "C" size_t st_trace_noalloc_scratch_bytes(void) { return kScratchBytes; }

extern "C" int st_trace_noalloc(st_scene *s, const st_camera *cam, const st_tiles *tl, const st_trace_opts *opts,
                                float *depth, float *normal, uint32_t *evals, uint8_t *flags, uint64_t *counters,
                                void *stream) {
  using namespace st;
  if (!s || !cam || !tl || !depth || !normal || !evals || !flags) {
    set_error("st_trace_noalloc: null argument");
    return ST_ERR_INVALID;
  }
  if (cam->width <= 0 || cam->height <= 0 || cam->width > 65535 || cam->height > 65535 ||
      !(cam->vfov_deg > 0.f && cam->vfov_deg < 180.f)) {
    set_error("st_trace_noalloc: invalid camera");
    return ST_ERR_INVALID;
  }
  if (tl->tile != 8 && tl->tile != 16 && tl->tile != 32) {
    set_error("st_trace_noalloc: tile must be 8, 16 or 32");
    return ST_ERR_INVALID;
  }
  const int tiles_x = (cam->width + tl->tile - 1) / tl->tile, tiles_y = (cam->height + tl->tile - 1) / tl->tile;
  if (tl->tiles_x != tiles_x || tl->tiles_y != tiles_y) {
    set_error("st_trace_noalloc: tile buffer does not match the camera");
    return ST_ERR_INVALID;
  }
  st_trace_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.step_mode != ST_STEP_PLAIN && o.step_mode != ST_STEP_OVERRELAX && o.step_mode != ST_STEP_LEARNED &&
      o.step_mode != ST_STEP_CROSSING) {
    set_error("st_trace_noalloc: unknown step mode");
    return ST_ERR_INVALID;
  }
  if (o.step_mode == ST_STEP_LEARNED && (!o.mlp || ((uintptr_t)o.mlp & 15u))) {
    set_error("st_trace_noalloc: ST_STEP_LEARNED needs opts.mlp: 16-byte aligned device pointer to packed MLP "
              "weights");
    return ST_ERR_INVALID;
  }
  unsigned char *scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != ST_OK) return rc;

  Job job;
  std::memset(&job, 0, sizeof(job));
  int stack_depth = 0, n_sm = 1;
  double diameter = 0, extent = 0;
  scene_facts(s, &job.sc, &stack_depth, &diameter, &extent, &n_sm);
  camera_basis(*cam, job.cam);
  job.tl.tile = tl->tile;
  job.tl.tiles_x = tl->tiles_x;
  job.tl.tiles_y = tl->tiles_y;
  job.tl.offsets = tl->offsets;
  job.tl.z_in = tl->z_in;
  job.tl.z_out = tl->z_out;
  job.tl.prim = tl->prim;
  job.out.depth = depth;
  job.out.normal = normal;
  job.out.evals = evals;
  job.out.flags = flags;
  job.tp = make_trace_params(o, diameter, extent);
  job.tile_base = 0;

  // The same launch as st_trace: parameter cache size, stack slots, work
  // area placement, longest-list-first tile order and split records.
  TraceLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.max_tile_rays = tl->tile * tl->tile;
  L.act_cap = (int)std::max<uint32_t>(tl->max_overlap, 1u);
  L.view_cap = 2 * L.act_cap;
  L.stack_slots = stack_depth + 2;
  L.dc_words = trace_dcache_words(L.view_cap, tl->max_overlap, tl->n_entries, n_sm);
  L.n_items = (uint32_t)(tiles_x * tiles_y);
  L.counters = counters;
  L.tile_stats = o.tile_stats;
  L.step_mode = job.tp.step_mode;
  L.further = scene_further_level(s);
  L.mlp = job.tp.step_mode == ST_STEP_LEARNED ? o.mlp : nullptr;
  if (job.tp.step_mode == ST_STEP_LEARNED && L.stack_slots < 10) L.stack_slots = 10;
  L.work_in_smem = 1;
  if (trace_smem_per_warp(L) * 16 > 200 * 1024) L.work_in_smem = 0;
  L.staged = trace_staged(L);
  L.prune_views = o.full_views ? 0 : 1;
  // (no CTA-split evaluation here: its per-CTA arrays would cut the lists
  // that fit the static scratch; it changes no output byte)

  const size_t order_off = (kJobOff + sizeof(Job) + 255) & ~size_t(255);
  const size_t work_off = (order_off + (size_t)L.n_items * 4 + 255) & ~size_t(255);
  if (work_off > kScratchBytes) {
    set_error("st_trace_noalloc: the tile order of " + std::to_string(L.n_items) + " tiles needs more than the " +
              "32 MiB static scratch; use st_trace");
    return ST_ERR_CAPACITY;
  }
  size_t work_end = work_off;
  if (!L.work_in_smem) {
    // One work area per resident CTA of the persistent grid (the kernel
    // indexes them by blockIdx.x).
    const int per_sm = trace_ctas_per_sm(L);
    if (per_sm < 1) {
      set_error("st_trace_noalloc: no valid launch configuration");
      return ST_ERR_INVALID;
    }
    L.g_work_words = trace_work_words(L);
    const size_t need = (size_t)n_sm * per_sm * L.g_work_words * 4;
    if (need > kScratchBytes - work_off) {
      set_error("st_trace_noalloc: the per-CTA work areas for tile lists of " + std::to_string(tl->max_overlap) +
                " entries need " + std::to_string(work_off + need) + " bytes, more than the 32 MiB static scratch; "
                "use st_trace");
      return ST_ERR_CAPACITY;
    }
    L.g_work = reinterpret_cast<uint32_t *>(scratch + work_off);
    work_end = work_off + need;
  }
  // Then the records of tiles split across CTAs, as many as fit.
  const long long split_cycles = trace_split_cycles(o.split_kcycles);
  const size_t split_off = (work_end + 255) & ~size_t(255);
  size_t used = work_end;
  if (split_cycles >= 0 && split_off < kScratchBytes) {
    uint32_t cap = trace_split_cap(L.max_tile_rays, L.n_items);
    const size_t room = (kScratchBytes - split_off) / 4;
    while (cap > 0 && trace_split_words(L.max_tile_rays, cap) > room) cap >>= 1;
    if (cap > 0) {
      L.split = reinterpret_cast<uint32_t *>(scratch + split_off);
      L.split_cap = cap;
      L.split_cycles = split_cycles;
      L.heavy_len = trace_heavy_len(o.heavy_split_len);
      used = split_off + trace_split_words(L.max_tile_rays, cap) * 4;
    }
  }
  L.idle_spins = o.wait_spin_limit;
  L.split_spins = o.wait_spin_limit;
  L.item_counter = reinterpret_cast<uint32_t *>(scratch + kCounterOff);
  uint32_t *status = reinterpret_cast<uint32_t *>(scratch + kStatusOff);
  if (o.check_status) L.status = status;
  uint32_t *order = reinterpret_cast<uint32_t *>(scratch + order_off);
  Job *job_dev = reinterpret_cast<Job *>(scratch + kJobOff);
  g_last_work_in_scratch.store(L.work_in_smem ? 0 : 1);
  g_last_used.store(used);
  g_last_split_cap.store(L.split ? L.split_cap : 0);

  cudaStream_t st = (cudaStream_t)stream;
  // The scratch keeps the previous call's contents: the queue counter, the
  // status word and the split area's counters must start at zero; the job
  // record, tile order, work areas and split records are fully rewritten
  // before they are read.
  NA_CK(cudaMemsetAsync(L.item_counter, 0, 8, st));   // queue counter and status word
  if (L.split) NA_CK(cudaMemsetAsync(L.split, 0, trace_split_zero_bytes(L.split_cap), st));
  count_launch(), k_put_job<<<1, 32, 0, st>>>(job, job_dev);
  NA_CK(cudaGetLastError());
  const uint32_t heavy_rank = L.split ? trace_heavy_rank(o.heavy_split_len, o.heavy_split_rank) : 0u;
  uint32_t *heavy_thr = heavy_rank ? reinterpret_cast<uint32_t *>(scratch + kHeavyOff) : nullptr;
  launch_tile_order(job_dev, 1, L.n_items, order, st, heavy_rank, trace_heavy_min(tl->n_entries, L.n_items),
                    heavy_thr);
  NA_CK(cudaGetLastError());
  L.order = order;
  L.heavy_thr = heavy_thr;
  NA_CK(trace_launch(job_dev, 1, L, n_sm, st));
  if (L.status) return trace_status_code(status, st, "st_trace_noalloc");
  return ST_OK;
}

extern "C" int st_trace_noalloc_last_layout(uint64_t *out) {
  if (!out) {
    st::set_error("st_trace_noalloc_last_layout: null argument");
    return ST_ERR_INVALID;
  }
  out[0] = g_last_work_in_scratch.load();
  out[1] = g_last_used.load();
  out[2] = g_last_split_cap.load();
  return ST_OK;
}
