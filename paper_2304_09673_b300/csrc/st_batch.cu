// st_batch.cu -- batched rendering of many scenes and the autotuner of the
// per-scene tile size and subfrustum parameters (include/st.h, "batched
// rendering of many scenes").
//
// A batch concatenates the primitive and tile index spaces of its scenes
// (Job::prim_base, Job::tile_base) so that each culling step is one launch
// over every scene, and tracing is one persistent k_trace launch whose CTAs
// pull (scene, tile) items from a single counter.  Buffers are sized once by
// a synchronised culling pass, with headroom; the launch sequence is then
// captured in a CUDA graph that every render replays.  Device-side capacity
// checks (k_check_capacity, and the per-tile list check in k_trace) set a
// status word instead of overrunning a buffer; the host re-plans on it.
#include <cctype>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "st_kernels.h"

namespace st {
void scene_facts(const st_scene *s, DevScene *sc, int *stack_depth, double *diameter, double *extent, int *n_sm);
bool scene_has_stri(const st_scene *s);
int scene_further_level(const st_scene *s);
TraceParams make_trace_params(const st_trace_opts &o, double diameter, double extent);
}  // namespace st

using namespace st;

namespace {

// ---- the tune cache file ------------------------------------------------------------
// {"st_autotune": 1, "entries": {"<key>": {"tile": 16, "max_new_per_turn": 24,
//  "depth_slab_frac": 0.05, "ms": 1.25}, ...}}
struct Json {
  const char *p, *e;
  void ws() {
    while (p < e && std::isspace((unsigned char)*p)) ++p;
  }
  bool lit(char c) {
    ws();
    if (p < e && *p == c) { ++p; return true; }
    return false;
  }
  bool str(std::string &s) {
    ws();
    if (p >= e || *p != '"') return false;
    ++p;
    s.clear();
    while (p < e && *p != '"') {
      if (*p == '\\' && p + 1 < e) ++p;
      s.push_back(*p++);
    }
    if (p >= e) return false;
    ++p;
    return true;
  }
  bool num(double &v) {
    ws();
    if (p >= e) return false;
    std::string t;
    while (p < e && (std::isdigit((unsigned char)*p) || *p == '-' || *p == '+' || *p == '.' || *p == 'e' || *p == 'E'))
      t.push_back(*p++);
    if (t.empty()) return false;
    char *end = nullptr;
    v = std::strtod(t.c_str(), &end);
    return end && *end == '\0';
  }
  bool skip() {   // any value
    ws();
    if (p >= e) return false;
    if (*p == '"') { std::string s; return str(s); }
    if (*p == '{' || *p == '[') {
      const char open = *p, close = open == '{' ? '}' : ']';
      ++p;
      if (lit(close)) return true;
      for (;;) {
        if (open == '{') {
          std::string k;
          if (!str(k) || !lit(':')) return false;
        }
        if (!skip()) return false;
        if (lit(',')) continue;
        return lit(close);
      }
    }
    for (const char *w : {"true", "false", "null"}) {
      const size_t n = std::strlen(w);
      if ((size_t)(e - p) >= n && std::strncmp(p, w, n) == 0) { p += n; return true; }
    }
    double v;
    return num(v);
  }
};

bool parse_tune(Json &j, st_tune &t) {
  if (!j.lit('{')) return false;
  t.tile = 16; t.max_new_per_turn = 32; t.depth_slab_frac = 0.05f; t.ms = 0.f;
  if (j.lit('}')) return true;
  for (;;) {
    std::string k;
    if (!j.str(k) || !j.lit(':')) return false;
    if (k == "tile" || k == "max_new_per_turn" || k == "depth_slab_frac" || k == "ms") {
      double v;
      if (!j.num(v)) return false;
      if (k == "tile") t.tile = (int32_t)v;
      else if (k == "max_new_per_turn") t.max_new_per_turn = (int32_t)v;
      else if (k == "depth_slab_frac") t.depth_slab_frac = (float)v;
      else t.ms = (float)v;
    } else if (!j.skip()) {
      return false;
    }
    if (j.lit(',')) continue;
    return j.lit('}');
  }
}

// Returns 1 on success, 0 when the file does not exist, -1 when malformed.
int read_cache(const char *path, std::map<std::string, st_tune> &out) {
  FILE *f = std::fopen(path, "rb");
  if (!f) return 0;
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, n);
  std::fclose(f);
  Json j{text.data(), text.data() + text.size()};
  if (!j.lit('{')) return -1;
  if (j.lit('}')) return 1;
  for (;;) {
    std::string k;
    if (!j.str(k) || !j.lit(':')) return -1;
    if (k == "entries") {
      if (!j.lit('{')) return -1;
      if (!j.lit('}')) {
        for (;;) {
          std::string key;
          st_tune t;
          if (!j.str(key) || !j.lit(':') || !parse_tune(j, t)) return -1;
          out[key] = t;
          if (j.lit(',')) continue;
          if (!j.lit('}')) return -1;
          break;
        }
      }
    } else if (!j.skip()) {
      return -1;
    }
    if (j.lit(',')) continue;
    return j.lit('}') ? 1 : -1;
  }
}

bool write_cache(const char *path, const std::map<std::string, st_tune> &m) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = std::fopen(tmp.c_str(), "wb");
  if (!f) return false;
  std::fprintf(f, "{\"st_autotune\": 1, \"entries\": {");
  bool first = true;
  for (const auto &kv : m) {
    std::fprintf(f, "%s\n  \"%s\": {\"tile\": %d, \"max_new_per_turn\": %d, \"depth_slab_frac\": %.9g, \"ms\": %.6g}",
                 first ? "" : ",", kv.first.c_str(), kv.second.tile, kv.second.max_new_per_turn,
                 (double)kv.second.depth_slab_frac, (double)kv.second.ms);
    first = false;
  }
  std::fprintf(f, "\n}}\n");
  const bool ok = std::fclose(f) == 0;
  return ok && std::rename(tmp.c_str(), path) == 0;
}

bool valid_tune(const st_tune &t) {
  return (t.tile == 8 || t.tile == 16 || t.tile == 32) && t.max_new_per_turn >= 1 && t.max_new_per_turn <= 1024 &&
         t.depth_slab_frac > 0.f && std::isfinite(t.depth_slab_frac);
}

#define BK(call)                                                          \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess) {                                              \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));      \
      return ST_ERR_CUDA;                                                 \
    }                                                                     \
  } while (0)

template <class T>
struct Buf {   // device buffer owned by a batch or the autotuner
  T *p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t n) {
    if (n <= cap) return cudaSuccess;
    release();
    count_device_alloc();
    cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e == cudaSuccess) cap = n; else p = nullptr;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

int camera_ok(const st_camera &c) {
  return c.width > 0 && c.height > 0 && c.width <= 65535 && c.height <= 65535 && c.vfov_deg > 0.f &&
         c.vfov_deg < 180.f;
}

}  // namespace

struct st_batch {
  std::vector<st_scene *> scenes;
  std::vector<st_camera> cams;
  std::vector<st_tune> tune;
  std::vector<float *> depth, normal;
  std::vector<uint32_t *> evals;
  std::vector<uint8_t *> flags;
  st_trace_opts opts;
  cudaStream_t stream = nullptr;       // caller's stream: sizing pass and replays
  cudaStream_t cap_stream = nullptr;   // private stream the graph is captured on
  int n_sm = 1;
  uint32_t n_prims = 0, n_tiles = 0;
  std::vector<Job> jobs;
  Buf<Job> d_jobs;
  Buf<uint32_t> cand_count, cand_off, tile_count, offsets, scan_sums, small, item_counter, status, g_work, order, split;
  Buf<int4> rects;
  Buf<Pair> pairs;
  Buf<uint64_t> keys, counters;
  Buf<float> ztmp, z_in, z_out;
  Buf<uint32_t> prim;
  uint32_t pair_cap = 0, overlap_cap = 0;
  uint32_t longest_seen = 0, entries_seen = 0;   // sizing pass: longest list, entry total
  bool has_stri = false;   // a scene holds rounded triangles (second culling launch)
  int further = 0;   // kernel instance tier: the largest scene_further_level of the scenes
  TraceLaunch L;
  int grid = 0;
  size_t smem = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t graph_kernels = 0;   // kernel launches captured in the graph
  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  }
};

namespace {

// small[0] candidate total, [1] pair counter, [2] longest list, [3] entry total
void enqueue_culling(st_batch *b, cudaStream_t s, uint32_t pair_cap) {
  uint32_t *cand_total = b->small.p + 0, *pair_counter = b->small.p + 1, *max_ov = b->small.p + 2,
           *tile_total = b->small.p + 3;
  cudaMemsetAsync(b->small.p, 0, 4 * sizeof(uint32_t), s);
  cudaMemsetAsync(b->tile_count.p, 0, (size_t)b->n_tiles * 4, s);
  launch_prim_bounds(b->d_jobs.p, (int)b->jobs.size(), b->n_prims, b->cand_count.p, b->rects.p, s);
  scan_u32(b->cand_count.p, b->cand_off.p, b->n_prims, b->scan_sums.p, cand_total, nullptr, nullptr, s);
  launch_cull_pairs(b->d_jobs.p, (int)b->jobs.size(), b->cand_off.p, b->n_prims, cand_total, b->rects.p,
                    b->tile_count.p, b->pairs.p, pair_cap, pair_counter, b->n_sm, s, b->has_stri);
  scan_u32(b->tile_count.p, b->offsets.p, b->n_tiles, b->scan_sums.p, tile_total, max_ov, b->offsets.p + b->n_tiles,
           s);
}

// Sizes and allocates every buffer, uploads the job table and captures the graph.
int plan(st_batch *b) {
  b->drop_graph();
  const int n = (int)b->scenes.size();
  b->jobs.assign(n, Job{});
  b->has_stri = false;
  b->further = 0;
  uint32_t prim_base = 0, tile_base = 0;
  int max_tile = 8, stack_slots = 2;
  for (int i = 0; i < n; ++i) {
    Job &j = b->jobs[i];
    std::memset(&j, 0, sizeof(Job));
    int sd = 0, nsm = 1;
    double diam = 0, ext = 0;
    scene_facts(b->scenes[i], &j.sc, &sd, &diam, &ext, &nsm);
    if (scene_has_stri(b->scenes[i])) b->has_stri = true;
    b->further = std::max(b->further, scene_further_level(b->scenes[i]));
    b->n_sm = nsm;
    camera_basis(b->cams[i], j.cam);
    const int T = b->tune[i].tile;
    j.tl.tile = T;
    j.tl.tiles_x = (b->cams[i].width + T - 1) / T;
    j.tl.tiles_y = (b->cams[i].height + T - 1) / T;
    st_trace_opts o = b->opts;
    o.max_new_per_turn = b->tune[i].max_new_per_turn;
    o.depth_slab_frac = b->tune[i].depth_slab_frac;
    j.tp = make_trace_params(o, diam, ext);
    j.out.depth = b->depth[i];
    j.out.normal = b->normal[i];
    j.out.evals = b->evals[i];
    j.out.flags = b->flags[i];
    j.prim_base = prim_base;
    j.tile_base = tile_base;
    prim_base += (uint32_t)j.sc.n_prims;
    tile_base += (uint32_t)(j.tl.tiles_x * j.tl.tiles_y);
    max_tile = std::max(max_tile, T);
    stack_slots = std::max(stack_slots, sd + 2);
  }
  b->n_prims = prim_base;
  b->n_tiles = tile_base;
  cudaStream_t s = b->stream;
  BK(b->d_jobs.ensure((size_t)n));
  BK(b->cand_count.ensure(b->n_prims));
  BK(b->cand_off.ensure(b->n_prims));
  BK(b->rects.ensure(b->n_prims));
  BK(b->tile_count.ensure(b->n_tiles));
  BK(b->offsets.ensure((size_t)b->n_tiles + 1));
  BK(b->order.ensure(b->n_tiles));
  BK(b->scan_sums.ensure(std::max(scan_block_count(b->n_prims), scan_block_count(b->n_tiles)) + 2));
  BK(b->small.ensure(16));
  BK(b->item_counter.ensure(1));
  BK(b->status.ensure(1));
  BK(b->counters.ensure(ST_NUM_COUNTERS));
  BK(cull_set_attributes());

  // ---- sizing pass (synchronised) ----
  BK(cudaMemcpyAsync(b->d_jobs.p, b->jobs.data(), sizeof(Job) * n, cudaMemcpyHostToDevice, s));
  uint32_t cap = (uint32_t)std::max<size_t>(b->pairs.cap, std::max<size_t>(4096, (size_t)b->n_prims * 8));
  uint32_t host_small[4] = {0, 0, 0, 0};
  for (int attempt = 0; attempt < 3; ++attempt) {
    BK(b->pairs.ensure(cap));
    enqueue_culling(b, s, cap);
    BK(cudaGetLastError());
    BK(cudaMemcpyAsync(host_small, b->small.p, sizeof(host_small), cudaMemcpyDeviceToHost, s));
    BK(cudaStreamSynchronize(s));
    if (host_small[1] <= cap) break;
    cap = host_small[1];
  }
  if (host_small[1] > cap) { set_error("st_batch: culling did not converge"); return ST_ERR_CAPACITY; }
  b->longest_seen = host_small[2];
  b->entries_seen = host_small[3];
  // Headroom for edits between renders.
  b->pair_cap = (uint32_t)std::min<uint64_t>(0xFFFFFFF0ull, (uint64_t)host_small[1] * 3 / 2 + 4096);
  b->overlap_cap = std::max<uint32_t>(host_small[2] + host_small[2] / 4 + 16, 64);
  BK(b->pairs.ensure(b->pair_cap));
  BK(b->keys.ensure((size_t)b->pair_cap + 1));
  BK(b->ztmp.ensure((size_t)b->pair_cap + 1));
  BK(b->z_in.ensure((size_t)b->pair_cap + 1));
  BK(b->z_out.ensure((size_t)b->pair_cap + 1));
  BK(b->prim.ensure((size_t)b->pair_cap + 1));
  for (int i = 0; i < n; ++i) {
    Job &j = b->jobs[i];
    j.tl.offsets = b->offsets.p + j.tile_base;
    j.tl.z_in = b->z_in.p;
    j.tl.z_out = b->z_out.p;
    j.tl.prim = b->prim.p;
  }
  BK(cudaMemcpyAsync(b->d_jobs.p, b->jobs.data(), sizeof(Job) * n, cudaMemcpyHostToDevice, s));

  // ---- the persistent trace launch ----
  TraceLaunch &L = b->L;
  std::memset(&L, 0, sizeof(L));
  L.max_tile_rays = max_tile * max_tile;
  L.act_cap = (int)b->overlap_cap;
  L.view_cap = 2 * L.act_cap;
  L.stack_slots = stack_slots;
  L.dc_words = trace_dcache_words(L.view_cap, b->longest_seen, b->entries_seen, b->n_sm);
  L.n_items = b->n_tiles;
  L.item_counter = b->item_counter.p;
  L.counters = b->counters.p;
  L.status = b->status.p;
  L.order = b->order.p;
  L.step_mode = b->opts.step_mode;
  L.further = b->further;
  L.mlp = L.step_mode == ST_STEP_LEARNED ? b->opts.mlp : nullptr;
  if (L.step_mode == ST_STEP_LEARNED && L.stack_slots < 10) L.stack_slots = 10;
  L.work_in_smem = trace_smem_per_warp(L) * 16 > 200 * 1024 ? 0 : 1;
  L.staged = trace_staged(L);
  L.cta_min_view = trace_cta_min_view(L, b->opts.cta_eval_min_view, false);
  L.prune_views = b->opts.full_views ? 0 : 1;
  if (!L.work_in_smem) {
    // one work area per CTA of the persistent grid (indexed by blockIdx.x)
    const int per_sm = trace_ctas_per_sm(L);
    if (per_sm < 1) { set_error("st_batch: no valid launch configuration"); return ST_ERR_INVALID; }
    L.g_work_words = trace_work_words(L);
    BK(b->g_work.ensure((size_t)b->n_sm * per_sm * L.g_work_words));
    L.g_work = b->g_work.p;
  }
  const long long split_cycles = trace_split_cycles(b->opts.split_kcycles);
  if (split_cycles >= 0) {
    L.split_cap = trace_split_cap(L.max_tile_rays, L.n_items);
    BK(b->split.ensure(trace_split_words(L.max_tile_rays, L.split_cap)));
    L.split = b->split.p;
    L.split_cycles = split_cycles;
    L.heavy_len = trace_heavy_len(b->opts.heavy_split_len);
    if (trace_heavy_rank(b->opts.heavy_split_len, b->opts.heavy_split_rank)) L.heavy_thr = b->small.p + 6;
  }
  L.idle_spins = b->opts.wait_spin_limit;
  L.split_spins = b->opts.wait_spin_limit;
  BK(trace_plan(L, b->n_sm, &b->grid, &b->smem));
  BK(cudaStreamSynchronize(s));

  // ---- capture (on the batch's own stream: the caller's may be the legacy
  // default stream, which cannot be captured) ----
  if (!b->cap_stream) BK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  cudaStream_t cs = b->cap_stream;
  const uint64_t k0 = launches_so_far();
  BK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaMemsetAsync(b->status.p, 0, 4, cs);
  cudaMemsetAsync(b->item_counter.p, 0, 4, cs);
  cudaMemsetAsync(b->counters.p, 0, ST_NUM_COUNTERS * sizeof(uint64_t), cs);
  if (L.split) cudaMemsetAsync(L.split, 0, trace_split_zero_bytes(L.split_cap), cs);
  enqueue_culling(b, cs, b->pair_cap);
  launch_check_capacity(b->small.p + 1, b->pair_cap, b->small.p + 2, b->overlap_cap, b->status.p, cs);
  launch_scatter_sort(b->pairs.p, b->small.p + 1, b->pair_cap, b->offsets.p, b->n_tiles, b->overlap_cap, b->keys.p,
                      b->ztmp.p, b->z_in.p, b->z_out.p, b->prim.p, b->n_sm, cs, b->status.p, b->tile_count.p,
                      b->small.p + 5);
  {
    const uint32_t heavy_rank = L.split ? trace_heavy_rank(b->opts.heavy_split_len, b->opts.heavy_split_rank) : 0u;
    uint32_t *heavy_thr = heavy_rank ? const_cast<uint32_t *>(L.heavy_thr) : nullptr;
    launch_tile_order(b->d_jobs.p, n, b->n_tiles, b->order.p, cs, heavy_rank,
                      trace_heavy_min(b->entries_seen, b->n_tiles), heavy_thr);
  }
  cudaError_t le = trace_launch_planned(b->d_jobs.p, n, L, b->grid, b->smem, cs);
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(cs, &g);
  if (le != cudaSuccess || ce != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    set_error(std::string("st_batch: graph capture failed: ") + cudaGetErrorString(le != cudaSuccess ? le : ce));
    return ST_ERR_CUDA;
  }
  b->graph = g;
  b->graph_kernels = launches_so_far() - k0;
  count_launches(0 - b->graph_kernels);   // counted on replay instead
  BK(cudaGraphInstantiate(&b->exec, g, 0));
  return ST_OK;
}

void destroy(st_batch *b) {
  if (!b) return;
  b->drop_graph();
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  b->d_jobs.release(); b->cand_count.release(); b->cand_off.release(); b->tile_count.release();
  b->offsets.release(); b->scan_sums.release(); b->small.release(); b->item_counter.release();
  b->status.release(); b->g_work.release(); b->order.release(); b->split.release(); b->rects.release(); b->pairs.release(); b->keys.release();
  b->counters.release(); b->ztmp.release(); b->z_in.release(); b->z_out.release(); b->prim.release();
  delete b;
}

}  // namespace

extern "C" {

int st_tune_key(int n_prims, int width, int height, int step_mode, char *key, int cap) {
  if (n_prims < 1 || width < 1 || height < 1 || !key || cap < 1) { set_error("st_tune_key: invalid arguments"); return ST_ERR_INVALID; }
  const int nb = (int)std::lround(std::log2((double)n_prims));
  const int w = std::snprintf(key, (size_t)cap, "m%d_n%d_%dx%d", step_mode, nb, width, height);
  if (w < 0 || w >= cap) { set_error("st_tune_key: key buffer too small"); return ST_ERR_INVALID; }
  return ST_OK;
}

int st_tune_load(const char *path, const char *key, st_tune *out) {
  if (!path || !key || !out) { set_error("st_tune_load: null argument"); return ST_ERR_INVALID; }
  std::map<std::string, st_tune> m;
  const int r = read_cache(path, m);
  if (r <= 0) { set_error(r == 0 ? "st_tune_load: no cache file" : "st_tune_load: malformed cache file"); return ST_ERR_INVALID; }
  auto it = m.find(key);
  if (it == m.end() || !valid_tune(it->second)) { set_error("st_tune_load: key not in cache"); return ST_ERR_INVALID; }
  *out = it->second;
  return ST_OK;
}

int st_tune_store(const char *path, const char *key, const st_tune *t) {
  if (!path || !key || !t || !valid_tune(*t)) { set_error("st_tune_store: invalid arguments"); return ST_ERR_INVALID; }
  for (const char *c = key; *c; ++c)
    if (*c == '"' || *c == '\\' || (unsigned char)*c < 0x20) { set_error("st_tune_store: bad key"); return ST_ERR_INVALID; }
  std::map<std::string, st_tune> m;
  if (read_cache(path, m) < 0) { set_error("st_tune_store: existing cache file is malformed"); return ST_ERR_INVALID; }
  m[key] = *t;
  if (!write_cache(path, m)) { set_error("st_tune_store: cannot write the cache file"); return ST_ERR_INVALID; }
  return ST_OK;
}

int st_autotune(st_scene *scene, const st_camera *cam, const st_trace_opts *opts, const char *cache_path,
                st_tune *out, void *stream) {
  if (!scene || !cam || !out || !camera_ok(*cam)) { set_error("st_autotune: invalid arguments"); return ST_ERR_INVALID; }
  st_trace_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t npx = (size_t)cam->width * cam->height;
  Buf<float> depth, normal;
  Buf<uint32_t> evals;
  Buf<uint8_t> flags;
  BK(depth.ensure(npx));
  BK(normal.ensure(npx * 3));
  BK(evals.ensure(npx));
  BK(flags.ensure(npx));
  cudaEvent_t e0, e1;
  BK(cudaEventCreate(&e0));
  BK(cudaEventCreate(&e1));
  const int tiles[3] = {8, 16, 32};
  const int news[3] = {16, 32, 64};
  const float slabs[2] = {0.05f, 0.15f};
  st_tune best{16, 24, 0.05f, INFINITY};
  int rc = ST_OK;
  for (int ti = 0; ti < 3 && rc == ST_OK; ++ti) {
    st_tiles tl;
    float tiles_ms = 0.f;
    for (int rep = 0; rep < 3 && rc == ST_OK; ++rep) {
      cudaEventRecord(e0, s);
      rc = st_build_tiles(scene, cam, tiles[ti], &tl, stream);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tiles_ms += 0.5f * ms;
    }
    if (rc != ST_OK) break;
    for (int ni = 0; ni < 3 && rc == ST_OK; ++ni) {
      for (int si = 0; si < 2 && rc == ST_OK; ++si) {
        st_trace_opts c = o;
        c.max_new_per_turn = news[ni];
        c.depth_slab_frac = slabs[si];
        c.tile_stats = nullptr;
        float tr = 0.f;
        for (int rep = 0; rep < 3 && rc == ST_OK; ++rep) {
          cudaEventRecord(e0, s);
          rc = st_trace(scene, cam, &tl, &c, depth.p, normal.p, evals.p, flags.p, nullptr, stream);
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) tr += 0.5f * ms;
        }
        if (rc == ST_OK && tiles_ms + tr < best.ms) best = st_tune{tiles[ti], news[ni], slabs[si], tiles_ms + tr};
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  depth.release(); normal.release(); evals.release(); flags.release();
  if (rc != ST_OK) return rc;
  if (cudaGetLastError() != cudaSuccess) { set_error("st_autotune: CUDA error while timing"); return ST_ERR_CUDA; }
  *out = best;
  if (cache_path) {
    DevScene sc;
    int sd = 0, nsm = 0;
    double diam = 0, ext = 0;
    scene_facts(scene, &sc, &sd, &diam, &ext, &nsm);
    char key[96];
    rc = st_tune_key(sc.n_prims, cam->width, cam->height, o.step_mode, key, (int)sizeof(key));
    if (rc == ST_OK) rc = st_tune_store(cache_path, key, &best);
  }
  return rc;
}

int st_batch_create(st_scene *const *scenes, const st_camera *cams, int n, const st_trace_opts *opts,
                    float *const *depth, float *const *normal, uint32_t *const *evals, uint8_t *const *flags,
                    const char *autotune_cache, st_batch **out, void *stream) {
  if (!out) { set_error("st_batch_create: null output"); return ST_ERR_INVALID; }
  *out = nullptr;
  if (n < 1 || !scenes || !cams || !depth || !normal || !evals || !flags) {
    set_error("st_batch_create: invalid arguments");
    return ST_ERR_INVALID;
  }
  st_trace_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.step_mode != ST_STEP_PLAIN && o.step_mode != ST_STEP_OVERRELAX && o.step_mode != ST_STEP_LEARNED &&
      o.step_mode != ST_STEP_CROSSING) {
    set_error("st_batch_create: unknown step mode");
    return ST_ERR_INVALID;
  }
  if (o.step_mode == ST_STEP_LEARNED && (!o.mlp || ((uintptr_t)o.mlp & 15u))) {
    set_error("st_batch_create: ST_STEP_LEARNED needs opts.mlp (16-byte aligned device pointer)");
    return ST_ERR_INVALID;
  }
  o.tile_stats = nullptr;
  st_batch *b = new (std::nothrow) st_batch();
  if (!b) { set_error("host allocation failed"); return ST_ERR_NOMEM; }
  b->opts = o;
  b->stream = (cudaStream_t)stream;
  for (int i = 0; i < n; ++i) {
    if (!scenes[i] || !camera_ok(cams[i]) || !depth[i] || !normal[i] || !evals[i] || !flags[i]) {
      set_error("st_batch_create: invalid scene, camera or output of entry " + std::to_string(i));
      destroy(b);
      return ST_ERR_INVALID;
    }
    b->scenes.push_back(scenes[i]);
    b->cams.push_back(cams[i]);
    b->depth.push_back(depth[i]);
    b->normal.push_back(normal[i]);
    b->evals.push_back(evals[i]);
    b->flags.push_back(flags[i]);
    st_tune t{16, o.max_new_per_turn > 0 ? std::min(o.max_new_per_turn, 1024) : 32,
              o.depth_slab_frac > 0.f ? o.depth_slab_frac : 0.05f, 0.f};
    if (autotune_cache) {
      DevScene sc;
      int sd = 0, nsm = 0;
      double diam = 0, ext = 0;
      scene_facts(scenes[i], &sc, &sd, &diam, &ext, &nsm);
      char key[96];
      int rc = st_tune_key(sc.n_prims, cams[i].width, cams[i].height, o.step_mode, key, (int)sizeof(key));
      if (rc == ST_OK && st_tune_load(autotune_cache, key, &t) != ST_OK)
        rc = st_autotune(scenes[i], &cams[i], &o, autotune_cache, &t, stream);
      if (rc != ST_OK) { destroy(b); return rc; }
    }
    b->tune.push_back(t);
  }
  const int rc = plan(b);
  if (rc != ST_OK) {
    cudaStreamSynchronize(b->stream);
    destroy(b);
    return rc;
  }
  *out = b;
  return ST_OK;
}

int st_batch_render(st_batch *b, uint64_t *counters) {
  if (!b || !b->exec) { set_error("st_batch_render: invalid batch"); return ST_ERR_INVALID; }
  for (int attempt = 0; attempt < 3; ++attempt) {
    BK(cudaGraphLaunch(b->exec, b->stream));
    count_launches(b->graph_kernels);
    uint32_t status = 0;
    BK(cudaMemcpyAsync(&status, b->status.p, 4, cudaMemcpyDeviceToHost, b->stream));
    if (counters)
      BK(cudaMemcpyAsync(counters, b->counters.p, ST_NUM_COUNTERS * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                         b->stream));
    BK(cudaStreamSynchronize(b->stream));
    if (!(status & ST_STATUS_CAPACITY)) return ST_OK;
    if (attempt == 2) break;
    const int rc = plan(b);   // edits outgrew the planned buffers
    if (rc != ST_OK) return rc;
  }
  set_error("st_batch_render: tile lists outgrew the batch buffers");
  return ST_ERR_CAPACITY;
}

int st_batch_graph_kernels(const st_batch *b) { return b ? (int)b->graph_kernels : 0; }

int st_batch_tiles(const st_batch *b, int i) {
  if (!b || i < 0 || i >= (int)b->tune.size()) return 0;
  return b->tune[i].tile;
}

void st_batch_destroy(st_batch *b) { destroy(b); }

int st_render_batch(st_scene *const *scenes, const st_camera *cams, int n, const st_trace_opts *opts,
                    float *const *depth, float *const *normal, uint32_t *const *evals, uint8_t *const *flags,
                    const char *autotune_cache, void *stream) {
  st_batch *b = nullptr;
  int rc = st_batch_create(scenes, cams, n, opts, depth, normal, evals, flags, autotune_cache, &b, stream);
  if (rc != ST_OK) return rc;
  rc = st_batch_render(b, nullptr);
  destroy(b);
  return rc;
}

}  // extern "C"
