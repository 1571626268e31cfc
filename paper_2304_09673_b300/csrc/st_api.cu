// st_api.cu -- the C ABI (include/st.h): scene objects, A-buffer build,
// tracing.  No C++ exception crosses the boundary; every CUDA failure becomes
// ST_ERR_CUDA with the runtime's message in st_last_error().
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "st_kernels.h"

namespace st {

int trace_common(st_scene *s, const st_camera *cam, const st_tiles *tl, const st_trace_opts &o, float *depth,
                 float *normal, uint32_t *evals, uint8_t *flags, uint64_t *counters, void *stream, float *records,
                 uint32_t rec_cap, uint32_t *rec_count, int rec_stride);
int trace_status_code(const uint32_t *status, cudaStream_t st, const char *who);
TraceParams make_trace_params(const st_trace_opts &o, double diameter, double extent);

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
static std::atomic<uint64_t> g_launches{0};
int count_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return 0;
}
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
static std::atomic<uint64_t> g_allocs{0};
void count_device_alloc() { g_allocs.fetch_add(1, std::memory_order_relaxed); }
uint64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

#define ST_CK(call)                                                        \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) {                                               \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));       \
      return ST_ERR_CUDA;                                                  \
    }                                                                      \
  } while (0)

// Growable device buffer.
template <class T>
struct DBuf {
  T *p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t n) {
    if (n <= cap) return cudaSuccess;
    size_t want = n + n / 4 + 16;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    count_device_alloc();
    cudaError_t e = cudaMalloc(&p, want * sizeof(T));
    if (e == cudaSuccess) cap = want;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

static int device_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

}  // namespace st

using namespace st;

struct st_scene {
  Prep prep;
  int n_nodes = 0, n_prims = 0;
  float voi_pad = 1e-5f;
  // scene arrays
  DBuf<uint32_t> blob, rec_off, prim_addr, blk, lift, prim_index;
  DBuf<float4> rec;
  DBuf<float> d_prim;
  // full-resolution A-buffer and per-pixel tracing (st_build_dexels / st_trace_dexels)
  DBuf<uint32_t> dx_count, dx_offsets, dx_prim, dx_small;
  DBuf<uint64_t> dx_keys;
  DBuf<float> dx_ztmp, dx_zin, dx_zout;
  DBuf<uint2> dx_act;
  // culling buffers
  DBuf<uint32_t> cand_count, cand_off, tile_count, offsets, scan_sums, small;  // small: counters
  DBuf<int4> rects;
  DBuf<Pair> pairs;
  DBuf<uint64_t> keys;
  DBuf<float> ztmp, z_in, z_out;
  DBuf<uint32_t> prim;
  DBuf<Job> job;
  // tracing
  DBuf<uint32_t> g_work, item_counter, order, split;
  // updates
  DBuf<float4> upd_words;
  DBuf<uint32_t> upd_index;
  int n_sm = 1;
  int last_tile = 0;
  uint32_t last_max_overlap = 0;
};

namespace st {

__global__ void k_update_words(const uint32_t *idx, const float4 *words, uint32_t n, float4 *rec) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rec[idx[i]] = words[i];
}

static DevScene dev_scene(const st_scene *s) {
  DevScene d;
  d.blob = s->blob.p;
  d.rec_off = s->rec_off.p;
  d.rec = s->rec.p;
  d.prim_addr = s->prim_addr.p;
  d.d_prim = s->d_prim.p;
  d.blk = s->blk.p;
  d.lift = s->lift.p;
  d.prim_index = s->prim_index.p;
  d.lift_levels = s->prep.lift_levels;
  d.n_nodes = s->n_nodes;
  d.n_prims = s->n_prims;
  d.stack_depth = s->prep.stack_depth;
  d.diameter = (float)s->prep.diameter;
  d.voi_pad = s->voi_pad;
  return d;
}

bool scene_has_stri(const st_scene *s) { return s->prep.has_stri; }
int scene_further_level(const st_scene *s) { return s->prep.further_level(); }

// Read-only facts of a scene for entry points defined in other files.
void scene_facts(const st_scene *s, DevScene *sc, int *stack_depth, double *diameter, double *extent, int *n_sm) {
  *sc = dev_scene(s);
  *stack_depth = s->prep.stack_depth;
  *diameter = s->prep.diameter;
  *extent = s->prep.extent;
  *n_sm = s->n_sm;
}

static int check_camera(const st_camera *cam) {
  if (!cam || cam->width <= 0 || cam->height <= 0 || cam->width > 65535 || cam->height > 65535 ||
      !(cam->vfov_deg > 0.f && cam->vfov_deg < 180.f)) {
    set_error("invalid camera");
    return ST_ERR_INVALID;
  }
  return ST_OK;
}

}  // namespace st

extern "C" {

const char *st_last_error(void) { return st::g_err.c_str(); }
const char *st_version(void) { return "st 0.1 (sm_103a)"; }
uint64_t st_kernel_launches(void) { return g_launches.load(); }
uint64_t st_device_allocations(void) { return g_allocs.load(); }

int st_scene_create(const st_scene_desc *desc, st_scene **out, void *stream) {
  if (!desc || !out) { set_error("null argument"); return ST_ERR_INVALID; }
  *out = nullptr;
  st_scene *s = new (std::nothrow) st_scene();
  if (!s) { set_error("host allocation failed"); return ST_ERR_NOMEM; }
  std::string err;
  int rc = prepare(*desc, s->prep, err);
  if (rc != ST_OK) { set_error(err); delete s; return rc; }
  if (s->prep.stack_depth + 1 > ST_MAX_STACK) {
    set_error("tree needs a deeper evaluation stack than ST_MAX_STACK");
    delete s;
    return ST_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  s->n_nodes = desc->n_nodes;
  s->n_prims = (int)s->prep.prim_addr.size();
  s->voi_pad = desc->voi_pad > 0.f ? desc->voi_pad : 1e-5f;
  s->n_sm = device_sms();
  const Prep &p = s->prep;
  size_t nw = p.rec.size() / 4;
  auto fail = [&](cudaError_t e) {
    set_error(std::string("st_scene_create: ") + cudaGetErrorString(e));
    st_scene_destroy(s);
    return ST_ERR_CUDA;
  };
  cudaError_t e;
  if ((e = s->blob.ensure(p.blob.size())) != cudaSuccess) return fail(e);
  if ((e = s->rec_off.ensure(p.rec_off.size())) != cudaSuccess) return fail(e);
  if ((e = s->rec.ensure(nw)) != cudaSuccess) return fail(e);
  if ((e = s->prim_addr.ensure(p.prim_addr.size())) != cudaSuccess) return fail(e);
  if ((e = s->d_prim.ensure(p.d_prim.size())) != cudaSuccess) return fail(e);
  if ((e = s->blk.ensure(p.blk.size())) != cudaSuccess) return fail(e);
  if ((e = s->lift.ensure(p.lift.size())) != cudaSuccess) return fail(e);
  if ((e = s->prim_index.ensure(p.prim_index.size())) != cudaSuccess) return fail(e);
  if ((e = s->small.ensure(16)) != cudaSuccess) return fail(e);
  if ((e = s->item_counter.ensure(4)) != cudaSuccess) return fail(e);
  if ((e = s->job.ensure(1)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpyAsync(s->blob.p, p.blob.data(), p.blob.size() * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpyAsync(s->rec_off.p, p.rec_off.data(), p.rec_off.size() * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpyAsync(s->rec.p, p.rec.data(), nw * 16, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpyAsync(s->prim_addr.p, p.prim_addr.data(), p.prim_addr.size() * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpyAsync(s->d_prim.p, p.d_prim.data(), p.d_prim.size() * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpyAsync(s->blk.p, p.blk.data(), p.blk.size() * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpyAsync(s->lift.p, p.lift.data(), p.lift.size() * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpyAsync(s->prim_index.p, p.prim_index.data(), p.prim_index.size() * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
  *out = s;
  return ST_OK;
}

void st_scene_destroy(st_scene *s) {
  if (!s) return;
  s->blob.release(); s->rec_off.release(); s->prim_addr.release(); s->rec.release(); s->d_prim.release();
  s->blk.release(); s->lift.release();
  s->cand_count.release(); s->cand_off.release(); s->tile_count.release(); s->offsets.release();
  s->scan_sums.release(); s->small.release(); s->rects.release(); s->pairs.release(); s->keys.release();
  s->ztmp.release(); s->z_in.release(); s->z_out.release(); s->prim.release(); s->job.release();
  s->g_work.release(); s->item_counter.release(); s->order.release(); s->split.release(); s->upd_words.release();
  s->upd_index.release(); s->prim_index.release();
  s->dx_count.release(); s->dx_offsets.release(); s->dx_prim.release(); s->dx_small.release();
  s->dx_keys.release(); s->dx_ztmp.release(); s->dx_zin.release(); s->dx_zout.release(); s->dx_act.release();
  delete s;
}

int st_scene_info(const st_scene *s, double *out) {
  if (!s || !out) { set_error("null argument"); return ST_ERR_INVALID; }
  out[0] = s->prep.diameter;
  out[1] = s->prep.extent;
  out[2] = (double)s->n_prims;
  out[3] = (double)s->prep.stack_depth;
  return ST_OK;
}

int st_scene_addresses(const st_scene *s, int32_t *po_of_desc) {
  if (!s || !po_of_desc) { set_error("null argument"); return ST_ERR_INVALID; }
  std::memcpy(po_of_desc, s->prep.po_of_desc.data(), s->prep.po_of_desc.size() * sizeof(int32_t));
  return ST_OK;
}

int st_scene_update_prims(st_scene *s, const int32_t *ids, const float *params, int n, void *stream) {
  if (!s || (n > 0 && (!ids || !params)) || n < 0) { set_error("invalid arguments"); return ST_ERR_INVALID; }
  if (n == 0) return ST_OK;
  std::vector<float> words;
  std::vector<uint32_t> index;
  words.reserve((size_t)n * 16);
  for (int i = 0; i < n; ++i) {
    int id = ids[i];
    if (id < 0 || id >= s->n_nodes) { set_error("node id out of range"); return ST_ERR_INVALID; }
    int a = s->prep.po_of_desc[id];
    uint32_t b = s->prep.blob[a];
    if (!blob_isprim(b)) { set_error("node id is not a primitive"); return ST_ERR_INVALID; }
    int kind = (int)blob_kind(b);
    if (const char *e = prim_record_error(kind, params + (size_t)i * ST_REC_FLOATS)) {
      set_error(std::string("st_scene_update_prims: ") + e);
      return ST_ERR_INVALID;
    }
    float w[4 * kMaxRecWords];
    prim_words(kind, params + (size_t)i * ST_REC_FLOATS, w);
    for (int k = 0; k < rec_words(kind); ++k) {
      index.push_back(s->prep.rec_off[a] + k);
      words.insert(words.end(), w + 4 * k, w + 4 * k + 4);
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t m = (uint32_t)index.size();
  ST_CK(s->upd_words.ensure(m));
  ST_CK(s->upd_index.ensure(m));
  ST_CK(cudaMemcpyAsync(s->upd_words.p, words.data(), (size_t)m * 16, cudaMemcpyHostToDevice, st));
  ST_CK(cudaMemcpyAsync(s->upd_index.p, index.data(), (size_t)m * 4, cudaMemcpyHostToDevice, st));
  count_launch(), k_update_words<<<(m + 255) / 256, 256, 0, st>>>(s->upd_index.p, s->upd_words.p, m, s->rec.p);
  ST_CK(cudaGetLastError());
  // The staging buffers are reused by the next call; keep host arrays alive
  // until the copies have been consumed.
  ST_CK(cudaStreamSynchronize(st));
  return ST_OK;
}

int st_build_tiles(st_scene *s, const st_camera *cam, int tile, st_tiles *out, void *stream) {
  if (!s || !out) { set_error("null argument"); return ST_ERR_INVALID; }
  int rc = check_camera(cam);
  if (rc != ST_OK) return rc;
  if (tile != 8 && tile != 16 && tile != 32) { set_error("tile must be 8, 16 or 32"); return ST_ERR_INVALID; }
  cudaStream_t st = (cudaStream_t)stream;
  const int tiles_x = (cam->width + tile - 1) / tile, tiles_y = (cam->height + tile - 1) / tile;
  const uint32_t n_tiles = (uint32_t)tiles_x * (uint32_t)tiles_y;
  const uint32_t np = (uint32_t)s->n_prims;

  static thread_local bool attr_done = false;
  if (!attr_done) { ST_CK(cull_set_attributes()); attr_done = true; }

  Job job;
  std::memset(&job, 0, sizeof(job));
  job.sc = dev_scene(s);
  camera_basis(*cam, job.cam);
  job.tl.tile = tile;
  job.tl.tiles_x = tiles_x;
  job.tl.tiles_y = tiles_y;
  ST_CK(s->cand_count.ensure(np));
  ST_CK(s->cand_off.ensure(np));
  ST_CK(s->rects.ensure(np));
  ST_CK(s->tile_count.ensure(n_tiles));
  ST_CK(s->offsets.ensure(n_tiles + 1));
  ST_CK(s->scan_sums.ensure(std::max(scan_block_count(np), scan_block_count(n_tiles)) + 2));
  if (s->pairs.cap == 0) ST_CK(s->pairs.ensure(std::max<size_t>(1024, (size_t)np * 8)));
  ST_CK(cudaMemcpyAsync(s->job.p, &job, sizeof(Job), cudaMemcpyHostToDevice, st));

  // small[0] candidate total, [1] pair counter, [2] longest list, [3] tile total
  uint32_t *cand_total = s->small.p + 0, *pair_counter = s->small.p + 1, *max_ov = s->small.p + 2,
           *tile_total = s->small.p + 3;
  launch_prim_bounds(s->job.p, 1, np, s->cand_count.p, s->rects.p, st);
  scan_u32(s->cand_count.p, s->cand_off.p, np, s->scan_sums.p, cand_total, nullptr, nullptr, st);
  uint32_t host_small[4] = {0, 0, 0, 0};
  for (int attempt = 0; attempt < 2; ++attempt) {
    ST_CK(cudaMemsetAsync(s->tile_count.p, 0, (size_t)n_tiles * 4, st));
    ST_CK(cudaMemsetAsync(s->small.p + 1, 0, 3 * sizeof(uint32_t), st));
    launch_cull_pairs(s->job.p, 1, s->cand_off.p, np, cand_total, s->rects.p, s->tile_count.p, s->pairs.p,
                      (uint32_t)s->pairs.cap, pair_counter, s->n_sm, st, s->prep.has_stri);
    scan_u32(s->tile_count.p, s->offsets.p, n_tiles, s->scan_sums.p, tile_total, max_ov,
             s->offsets.p + n_tiles, st);
    ST_CK(cudaGetLastError());
    ST_CK(cudaMemcpyAsync(host_small, s->small.p, sizeof(host_small), cudaMemcpyDeviceToHost, st));
    ST_CK(cudaStreamSynchronize(st));
    if (host_small[1] <= s->pairs.cap) break;
    ST_CK(s->pairs.ensure(host_small[1]));  // on-demand growth, then redo (Sec. 10)
  }
  const uint32_t n_entries = host_small[1];
  const uint32_t max_overlap = host_small[2];
  ST_CK(s->keys.ensure(n_entries + 1));
  ST_CK(s->ztmp.ensure(n_entries + 1));
  ST_CK(s->z_in.ensure(n_entries + 1));
  ST_CK(s->z_out.ensure(n_entries + 1));
  ST_CK(s->prim.ensure(n_entries + 1));
  // (tile_count is free after the scan: it lists the tiles of lists longer
  // than the shared-memory sort, counted in small[5])
  launch_scatter_sort(s->pairs.p, pair_counter, (uint32_t)s->pairs.cap, s->offsets.p, n_tiles, max_overlap,
                      s->keys.p, s->ztmp.p, s->z_in.p, s->z_out.p, s->prim.p, s->n_sm, st, nullptr,
                      s->tile_count.p, s->small.p + 5);
  ST_CK(cudaGetLastError());
  out->tile = tile;
  out->tiles_x = tiles_x;
  out->tiles_y = tiles_y;
  out->offsets = s->offsets.p;
  out->z_in = s->z_in.p;
  out->z_out = s->z_out.p;
  out->prim = s->prim.p;
  out->n_entries = n_entries;
  out->max_overlap = max_overlap;
  s->last_tile = tile;
  s->last_max_overlap = max_overlap;
  return ST_OK;
}

int st_trace(st_scene *s, const st_camera *cam, const st_tiles *tl, const st_trace_opts *opts, float *depth,
             float *normal, uint32_t *evals, uint8_t *flags, uint64_t *counters, void *stream) {
  if (!s || !tl || !depth || !normal || !evals || !flags) { set_error("null argument"); return ST_ERR_INVALID; }
  int rc = check_camera(cam);
  if (rc != ST_OK) return rc;
  const int tiles_x = (cam->width + tl->tile - 1) / tl->tile, tiles_y = (cam->height + tl->tile - 1) / tl->tile;
  if (tl->tiles_x != tiles_x || tl->tiles_y != tiles_y) {
    set_error("tile buffer does not match the camera");
    return ST_ERR_INVALID;
  }
  st_trace_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.step_mode != ST_STEP_PLAIN && o.step_mode != ST_STEP_OVERRELAX && o.step_mode != ST_STEP_LEARNED &&
      o.step_mode != ST_STEP_CROSSING) {
    set_error("unknown step mode");
    return ST_ERR_INVALID;
  }
  if (o.step_mode == ST_STEP_LEARNED && (!o.mlp || ((uintptr_t)o.mlp & 15u))) {
    set_error("ST_STEP_LEARNED needs opts.mlp: 16-byte aligned device pointer to packed MLP weights");
    return ST_ERR_INVALID;
  }
  return trace_common(s, cam, tl, o, depth, normal, evals, flags, counters, stream, nullptr, 0, nullptr, 0);
}

int st_trace_record(st_scene *s, const st_camera *cam, const st_tiles *tl, const st_trace_opts *opts,
                    float *depth, float *normal, uint32_t *evals, uint8_t *flags, float *records,
                    uint32_t rec_cap, uint32_t *rec_count, int ray_stride, void *stream) {
  if (!s || !tl || !depth || !normal || !evals || !flags || !records || !rec_count || ray_stride < 1) {
    set_error("st_trace_record: invalid arguments");
    return ST_ERR_INVALID;
  }
  int rc = check_camera(cam);
  if (rc != ST_OK) return rc;
  st_trace_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  o.step_mode = ST_STEP_RECORD;
  return trace_common(s, cam, tl, o, depth, normal, evals, flags, nullptr, stream, records, rec_cap, rec_count,
                      ray_stride);
}

}  // extern "C"

namespace st {

// Trace parameters of st_trace_opts, with the documented defaults.
TraceParams make_trace_params(const st_trace_opts &o, double diameter, double extent) {
  TraceParams tp;
  tp.eps = o.eps > 0.f ? o.eps : 1e-4f;
  tp.lipschitz = o.lipschitz > 0.f ? o.lipschitz : 1.45f;
  tp.max_steps = o.max_steps > 0 ? o.max_steps : 256;
  tp.step_mode = o.step_mode;
  const float frac = o.depth_slab_frac > 0.f ? o.depth_slab_frac : 0.05f;
  tp.depth_slab = std::max(frac * (float)diameter, 1e-6f);
  tp.max_new = o.max_new_per_turn > 0 ? std::min(o.max_new_per_turn, 1024) : 32;
  tp.newton_iters = o.newton_iters > 0 ? o.newton_iters : (o.newton_iters < 0 ? 0 : 2);
  tp.newton_clamp = o.newton_clamp > 0.f ? o.newton_clamp : 64.f * tp.eps;
  tp.omega = o.omega > 1.f ? std::min(o.omega, 2.f) : 1.7f;
  tp.min_step = o.min_step > 0.f ? o.min_step : std::max((float)(extent / 32000.0), 1e-7f);
  return tp;
}

int trace_common(st_scene *s, const st_camera *cam, const st_tiles *tl, const st_trace_opts &o, float *depth,
                 float *normal, uint32_t *evals, uint8_t *flags, uint64_t *counters, void *stream, float *records,
                 uint32_t rec_cap, uint32_t *rec_count, int rec_stride) {
  const int tiles_x = (cam->width + tl->tile - 1) / tl->tile, tiles_y = (cam->height + tl->tile - 1) / tl->tile;
  if (tl->tiles_x != tiles_x || tl->tiles_y != tiles_y) {
    set_error("tile buffer does not match the camera");
    return ST_ERR_INVALID;
  }
  Job job;
  std::memset(&job, 0, sizeof(job));
  job.sc = dev_scene(s);
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
  TraceParams &tp = job.tp;
  tp = make_trace_params(o, s->prep.diameter, s->prep.extent);
  job.tile_base = 0;
  cudaStream_t st = (cudaStream_t)stream;

  TraceLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.max_tile_rays = tl->tile * tl->tile;
  L.act_cap = (int)std::max<uint32_t>(tl->max_overlap, 1u);
  L.view_cap = 2 * L.act_cap;
  L.stack_slots = s->prep.stack_depth + 2;
  L.dc_words = trace_dcache_words(L.view_cap, tl->max_overlap, tl->n_entries, s->n_sm);
  L.n_items = (uint32_t)(tiles_x * tiles_y);
  L.counters = counters;
  L.tile_stats = o.tile_stats;
  L.step_mode = tp.step_mode;
  L.further = s->prep.further_level();
  L.mlp = tp.step_mode == ST_STEP_LEARNED ? o.mlp : nullptr;
  L.records = records;
  L.rec_cap = rec_cap;
  L.rec_count = rec_count;
  L.rec_stride = rec_stride > 0 ? rec_stride : 1;
  if (tp.step_mode == ST_STEP_LEARNED && L.stack_slots < 10) L.stack_slots = 10;
  // Active set and view in shared memory when 16 warps per SM still fit.
  L.work_in_smem = 1;
  if (trace_smem_per_warp(L) * 16 > 200 * 1024) L.work_in_smem = 0;
  L.staged = trace_staged(L);
  L.cta_min_view = trace_cta_min_view(L, o.cta_eval_min_view, true);
  L.prune_views = o.full_views ? 0 : 1;
  if (!L.work_in_smem) {
    // one work area per CTA of the persistent grid (indexed by blockIdx.x)
    const int per_sm = trace_ctas_per_sm(L);
    if (per_sm < 1) { set_error("st_trace: no valid launch configuration"); return ST_ERR_INVALID; }
    L.g_work_words = trace_work_words(L);
    ST_CK(s->g_work.ensure((size_t)s->n_sm * per_sm * L.g_work_words));
    L.g_work = s->g_work.p;
  }
  ST_CK(s->item_counter.ensure(4));
  L.item_counter = s->item_counter.p;
  ST_CK(s->job.ensure(1));
  ST_CK(cudaMemcpyAsync(s->job.p, &job, sizeof(Job), cudaMemcpyHostToDevice, st));
  ST_CK(cudaMemsetAsync(s->item_counter.p, 0, 4, st));
  ST_CK(s->order.ensure(L.n_items));
  const long long split_cycles = trace_split_cycles(o.split_kcycles);
  const uint32_t heavy_rank = split_cycles >= 0 && tp.step_mode != ST_STEP_RECORD
                                  ? trace_heavy_rank(o.heavy_split_len, o.heavy_split_rank) : 0u;
  uint32_t *heavy_thr = heavy_rank ? s->small.p + 9 : nullptr;
  launch_tile_order(s->job.p, 1, L.n_items, s->order.p, st, heavy_rank, trace_heavy_min(tl->n_entries, L.n_items),
                    heavy_thr);
  L.order = s->order.p;
  L.heavy_thr = heavy_thr;
  if (split_cycles >= 0 && tp.step_mode != ST_STEP_RECORD) {
    L.split_cap = trace_split_cap(L.max_tile_rays, L.n_items);
    ST_CK(s->split.ensure(trace_split_words(L.max_tile_rays, L.split_cap)));
    L.split = s->split.p;
    L.split_cycles = split_cycles;
    L.heavy_len = trace_heavy_len(o.heavy_split_len);
    ST_CK(cudaMemsetAsync(L.split, 0, trace_split_zero_bytes(L.split_cap), st));
  }
  L.idle_spins = o.wait_spin_limit;
  L.split_spins = o.wait_spin_limit;
  uint32_t *status = o.check_status ? s->small.p + 8 : nullptr;
  if (status) {
    ST_CK(cudaMemsetAsync(status, 0, sizeof(uint32_t), st));
    L.status = status;
  }
  ST_CK(trace_launch(s->job.p, 1, L, s->n_sm, st));
  if (status) return trace_status_code(status, st, "st_trace");
  return ST_OK;
}

// Reads a launch's device status word (synchronising the stream) and maps
// its bits to a return code: a bounded wait that ran out -> ST_ERR_TIMEOUT;
// a list beyond the launch's capacity -> ST_ERR_CAPACITY; a view or stack
// overflow -> ST_ERR_INVALID.
int trace_status_code(const uint32_t *status, cudaStream_t st, const char *who) {
  uint32_t h = 0;
  ST_CK(cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, st));
  ST_CK(cudaStreamSynchronize(st));
  if (h & ST_STATUS_WAIT) {
    set_error(std::string(who) + ": a bounded wait between the warps of a tile ran out (device status bit 3)");
    return ST_ERR_TIMEOUT;
  }
  if (h & ST_STATUS_CAPACITY) {
    set_error(std::string(who) + ": a tile list is longer than the launch's capacity (device status bit 2)");
    return ST_ERR_CAPACITY;
  }
  if (h & (ST_STATUS_VIEW | ST_STATUS_STACK)) {
    set_error(std::string(who) + ": a pruned view or evaluation stack overflowed (device status bits 0-1)");
    return ST_ERR_INVALID;
  }
  return ST_OK;
}

}  // namespace st

extern "C" {

static int pruned_view_common(const st_scene *s, const uint32_t *act, int n, uint32_t *view, uint32_t *view_addr,
                              int32_t *info, void *stream, int method) {
  if (!s || !act || n < 1 || n > s->n_prims || !view || !info) { set_error("invalid arguments"); return ST_ERR_INVALID; }
  cudaStream_t st = (cudaStream_t)stream;
  st_scene *m = const_cast<st_scene *>(s);
  const int cap = ST_MAX_STACK + 2;
  ST_CK(m->g_work.ensure(pruned_view_scratch_words(n, cap)));
  launch_pruned_view(dev_scene(s), act, n, view, view_addr, info, m->g_work.p, cap, method, st);
  ST_CK(cudaGetLastError());
  return ST_OK;
}

int st_pruned_view(const st_scene *s, const uint32_t *act, int n, uint32_t *view, uint32_t *view_addr,
                   int32_t *info, void *stream) {
  return pruned_view_common(s, act, n, view, view_addr, info, stream, 0);
}

int st_pruned_view_alg1(const st_scene *s, const uint32_t *act, int n, uint32_t *view, uint32_t *view_addr,
                        int32_t *info, void *stream) {
  return pruned_view_common(s, act, n, view, view_addr, info, stream, 1);
}

int st_pruned_view_live(const st_scene *s, const uint32_t *act, int n, uint32_t *view, uint32_t *view_addr,
                        int32_t *info, void *stream) {
  return pruned_view_common(s, act, n, view, view_addr, info, stream, 2);
}

int st_eval_pruned(const st_scene *s, const uint32_t *view, const int32_t *info, const float *pts, int npts,
                   float *f, float *grad, void *stream) {
  if (!s || !view || !info || (npts > 0 && (!pts || !f)) || npts < 0) { set_error("invalid arguments"); return ST_ERR_INVALID; }
  launch_eval_view(dev_scene(s), view, info, pts, npts, f, grad, (cudaStream_t)stream);
  ST_CK(cudaGetLastError());
  return ST_OK;
}

int st_eval_pruned_levels(const st_scene *s, const uint32_t *act, int n, uint32_t *view, int32_t *info,
                          const float *pts, int npts, float *f, void *stream) {
  if (!s || !act || n < 1 || n > s->n_prims || !view || !info || npts < 0 || (npts > 0 && (!pts || !f))) {
    set_error("invalid arguments");
    return ST_ERR_INVALID;
  }
  st_scene *m = const_cast<st_scene *>(s);
  const int cap = ST_MAX_STACK + 2;
  ST_CK(m->g_work.ensure(eval_levels_scratch_words(n, cap)));
  launch_eval_levels(dev_scene(s), act, n, view, info, m->g_work.p, cap, pts, npts, f, (cudaStream_t)stream);
  ST_CK(cudaGetLastError());
  return ST_OK;
}

int st_build_dexels(st_scene *s, const st_camera *cam, const st_tiles *tl, st_tiles *out, void *stream) {
  if (!s || !tl || !out) { set_error("null argument"); return ST_ERR_INVALID; }
  int rc = check_camera(cam);
  if (rc != ST_OK) return rc;
  if (tl->tile != 8 && tl->tile != 16 && tl->tile != 32) { set_error("tile lists must have tile 8, 16 or 32"); return ST_ERR_INVALID; }
  const int tiles_x = (cam->width + tl->tile - 1) / tl->tile, tiles_y = (cam->height + tl->tile - 1) / tl->tile;
  if (tl->tiles_x != tiles_x || tl->tiles_y != tiles_y) {
    set_error("tile buffer does not match the camera");
    return ST_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t n_pix = (uint32_t)cam->width * (uint32_t)cam->height;
  static thread_local bool attr_done = false;
  if (!attr_done) { ST_CK(cull_set_attributes()); attr_done = true; }
  Job job;
  std::memset(&job, 0, sizeof(job));
  job.sc = dev_scene(s);
  camera_basis(*cam, job.cam);
  job.tl.tile = tl->tile;
  job.tl.tiles_x = tl->tiles_x;
  job.tl.tiles_y = tl->tiles_y;
  job.tl.offsets = tl->offsets;
  job.tl.z_in = tl->z_in;
  job.tl.z_out = tl->z_out;
  job.tl.prim = tl->prim;
  ST_CK(s->dx_count.ensure(n_pix));
  ST_CK(s->dx_offsets.ensure((size_t)n_pix + 1));
  ST_CK(s->dx_small.ensure(4));
  ST_CK(s->scan_sums.ensure(scan_block_count(n_pix) + 2));
  ST_CK(cudaMemsetAsync(s->dx_small.p, 0, 4 * sizeof(uint32_t), st));
  launch_dexel_pass(job, false, s->dx_count.p, nullptr, nullptr, nullptr, st);
  scan_u32(s->dx_count.p, s->dx_offsets.p, n_pix, s->scan_sums.p, s->dx_small.p, s->dx_small.p + 1,
           s->dx_offsets.p + n_pix, st);
  ST_CK(cudaGetLastError());
  uint32_t host_small[2] = {0, 0};
  ST_CK(cudaMemcpyAsync(host_small, s->dx_small.p, sizeof(host_small), cudaMemcpyDeviceToHost, st));
  ST_CK(cudaStreamSynchronize(st));
  const uint32_t n_entries = host_small[0], max_len = host_small[1];
  ST_CK(s->dx_keys.ensure((size_t)n_entries + 1));
  ST_CK(s->dx_ztmp.ensure((size_t)n_entries + 1));
  ST_CK(s->dx_zin.ensure((size_t)n_entries + 1));
  ST_CK(s->dx_zout.ensure((size_t)n_entries + 1));
  ST_CK(s->dx_prim.ensure((size_t)n_entries + 1));
  launch_dexel_pass(job, true, nullptr, s->dx_offsets.p, s->dx_keys.p, s->dx_ztmp.p, st);
  launch_segment_sort(s->dx_offsets.p, n_pix, max_len, s->dx_keys.p, s->dx_ztmp.p, s->dx_zin.p, s->dx_zout.p,
                      s->dx_prim.p, s->n_sm, st);
  ST_CK(cudaGetLastError());
  out->tile = 1;
  out->tiles_x = cam->width;
  out->tiles_y = cam->height;
  out->offsets = s->dx_offsets.p;
  out->z_in = s->dx_zin.p;
  out->z_out = s->dx_zout.p;
  out->prim = s->dx_prim.p;
  out->n_entries = n_entries;
  out->max_overlap = max_len;
  return ST_OK;
}

int st_trace_dexels(st_scene *s, const st_camera *cam, const st_tiles *dx, const st_trace_opts *opts, int traversal,
                    float *depth, float *normal, uint32_t *evals, uint8_t *flags, uint64_t *counters, void *stream) {
  if (!s || !dx || !depth || !normal || !evals || !flags) { set_error("null argument"); return ST_ERR_INVALID; }
  int rc = check_camera(cam);
  if (rc != ST_OK) return rc;
  if (dx->tile != 1 || dx->tiles_x != cam->width || dx->tiles_y != cam->height) {
    set_error("st_trace_dexels: the dexel buffer (tile 1) does not match the camera");
    return ST_ERR_INVALID;
  }
  if (traversal != ST_TRAVERSE_PARENT && traversal != ST_TRAVERSE_FAST) {
    set_error("st_trace_dexels: unknown traversal");
    return ST_ERR_INVALID;
  }
  st_trace_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.step_mode != ST_STEP_PLAIN) {
    set_error("st_trace_dexels: only ST_STEP_PLAIN");
    return ST_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Job job;
  std::memset(&job, 0, sizeof(job));
  job.sc = dev_scene(s);
  camera_basis(*cam, job.cam);
  job.out.depth = depth;
  job.out.normal = normal;
  job.out.evals = evals;
  job.out.flags = flags;
  job.tp = make_trace_params(o, s->prep.diameter, s->prep.extent);
  int grid = 0;
  ST_CK(dexel_trace_grid(traversal == ST_TRAVERSE_FAST, s->n_sm, &grid));
  DexelLaunch D;
  std::memset(&D, 0, sizeof(D));
  D.offsets = dx->offsets;
  D.z_in = dx->z_in;
  D.z_out = dx->z_out;
  D.prim = dx->prim;
  D.n_threads = (uint32_t)grid * 128u;
  ST_CK(s->dx_act.ensure((size_t)std::max<uint32_t>(dx->max_overlap, 1u) * D.n_threads));
  D.act = s->dx_act.p;
  ST_CK(s->item_counter.ensure(4));
  D.pixel_counter = s->item_counter.p;
  D.counters = counters;
  ST_CK(cudaMemsetAsync(D.pixel_counter, 0, 4, st));
  ST_CK(launch_trace_dexel(job, D, traversal == ST_TRAVERSE_FAST, grid, st));
  return ST_OK;
}

int st_eval_sparse(const st_scene *s, const uint32_t *act, int n, const float *pts, int npts, int traversal, float *f,
                   uint32_t *status, void *stream) {
  if (!s || !act || n < 1 || n > s->n_prims || npts < 0 || (npts > 0 && (!pts || !f)) || !status) {
    set_error("invalid arguments");
    return ST_ERR_INVALID;
  }
  if (traversal != ST_TRAVERSE_PARENT && traversal != ST_TRAVERSE_FAST) { set_error("unknown traversal"); return ST_ERR_INVALID; }
  ST_CK(launch_eval_sparse(dev_scene(s), act, n, pts, npts, traversal == ST_TRAVERSE_FAST, f, status,
                           (cudaStream_t)stream));
  return ST_OK;
}

int st_tiles_copy(const st_tiles *t, uint32_t *offsets, float *z_in, float *z_out, uint32_t *prim,
                  void *stream) {
  if (!t) { set_error("null argument"); return ST_ERR_INVALID; }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nt = (size_t)t->tiles_x * t->tiles_y + 1, ne = (size_t)t->n_entries;
  if (offsets) ST_CK(cudaMemcpyAsync(offsets, t->offsets, nt * 4, cudaMemcpyDefault, st));
  if (ne && z_in) ST_CK(cudaMemcpyAsync(z_in, t->z_in, ne * 4, cudaMemcpyDefault, st));
  if (ne && z_out) ST_CK(cudaMemcpyAsync(z_out, t->z_out, ne * 4, cudaMemcpyDefault, st));
  if (ne && prim) ST_CK(cudaMemcpyAsync(prim, t->prim, ne * 4, cudaMemcpyDefault, st));
  ST_CK(cudaStreamSynchronize(st));
  return ST_OK;
}

}  // extern "C"
