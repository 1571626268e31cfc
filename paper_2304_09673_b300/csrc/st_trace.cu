// st_trace.cu -- synchronized sphere tracing of screen tiles (Sec. 8,
// Algorithm 2) over pruned tree views built by the sparse bottom-up traversal
// (Sec. 7, Algorithm 1, with the usage bits of Sec. 9) and evaluated by
// Algorithm 3.
//
// Execution model (own design for sm_103a):
//   * persistent CTAs of kWarps warps; every warp is an independent tile
//     worker pulling (job, tile) items from a global queue;
//   * per tile, the warp walks the depth-sorted A-buffer list, segmenting the
//     tile frustum into subfrustums [z_begin, z_end] with a fixed active
//     primitive set (Sec. 8 "tracking active primitives"; discard, fetch and
//     sorted merge are warp-parallel);
//   * one lane rebuilds the pruned view from the active set (Algorithm 1 with
//     fast ancestor pointers, clamping and popRequiredA / popRequiredB);
//   * all lanes then sphere-trace the subfrustum in lockstep over the same
//     view (warp-uniform node sequence, no divergence in the interpreter);
//     a lane whose ray hits, leaves the subfrustum or reaches the step cap
//     immediately takes the next pending ray of the tile (compaction of
//     finished rays), so lanes stay busy until the tile's queue drains;
//   * hits are refined with Newton steps on the ray (dual numbers) and get
//     the normalised forward-mode gradient of f_A as normal.
#include <cstdint>

#include "st_field.cuh"
#include "st_geom.cuh"
#include "st_kernels.h"

namespace st {

constexpr int kWarps = 4;

int trace_warps_per_cta() { return kWarps; }

enum RayStatus : uint32_t { R_ALIVE = 0, R_HIT = 1, R_UNCONV = 2 };

// Per-warp working set.  Shared memory always holds the ray state, queues and
// the evaluation stack; the active set and the view live either in shared
// memory or in a global per-warp region (long tile lists).
struct WarpWork {
  float *ray_z;          // [max_tile_rays] current depth of each ray
  uint32_t *ray_st;      // [max_tile_rays] steps | status << 24
  uint16_t *alive;       // [max_tile_rays] tile-local ids of pending rays
  uint16_t *hits;        // [max_tile_rays] rays that hit in this subfrustum
  float *stk;            // [stack_slots][32]
  uint32_t *bstk;        // [stack_slots + 2] Algorithm 1 stack (anc | usage << 31)
  uint32_t *act[2];      // [act_cap] active primitive addresses (sorted)
  float *act_ze[2];      // [act_cap] their exit depths
  uint32_t *view;        // [view_cap]
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline size_t smem_fixed_bytes(const TraceLaunch &L) {
  size_t r = (size_t)L.max_tile_rays;
  return align16(r * 4) + align16(r * 4) + align16(r * 2) + align16(r * 2) +
         align16((size_t)L.stack_slots * 32 * 4) + align16((size_t)(L.stack_slots + 2) * 4);
}
__host__ __device__ inline size_t work_bytes(const TraceLaunch &L) {
  return align16((size_t)L.act_cap * 4) * 4 + align16((size_t)L.view_cap * 4);
}

__host__ __device__ inline size_t smem_per_warp(const TraceLaunch &L) {
  return smem_fixed_bytes(L) + (L.work_in_smem ? work_bytes(L) : 0);
}
size_t trace_smem_per_warp(const TraceLaunch &L) { return smem_per_warp(L); }
uint32_t trace_work_words(const TraceLaunch &L) { return (uint32_t)(work_bytes(L) / 4); }

__device__ WarpWork carve(unsigned char *p, const TraceLaunch &L, uint32_t *gwork) {
  WarpWork w;
  size_t r = (size_t)L.max_tile_rays;
  w.ray_z = (float *)p; p += align16(r * 4);
  w.ray_st = (uint32_t *)p; p += align16(r * 4);
  w.alive = (uint16_t *)p; p += align16(r * 2);
  w.hits = (uint16_t *)p; p += align16(r * 2);
  w.stk = (float *)p; p += align16((size_t)L.stack_slots * 32 * 4);
  w.bstk = (uint32_t *)p; p += align16((size_t)(L.stack_slots + 2) * 4);
  unsigned char *q = L.work_in_smem ? p : (unsigned char *)gwork;
  size_t a = align16((size_t)L.act_cap * 4);
  w.act[0] = (uint32_t *)q; q += a;
  w.act[1] = (uint32_t *)q; q += a;
  w.act_ze[0] = (float *)q; q += a;
  w.act_ze[1] = (float *)q; q += a;
  w.view = (uint32_t *)q;
  return w;
}

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

__device__ ViewInfo build_view(const DevScene &sc, const uint32_t *act, int n, uint32_t *view,
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
      const uint32_t code = blob_kind(nb);  // primitive kinds equal their view codes
      if (vaddr) vaddr[nv] = P;
      view[nv++] = (code << kViewOffBits) | __ldg(sc.rec_off + P);
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
          view[nv++] = (code << kViewOffBits) | __ldg(sc.rec_off + pop);
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

// ---- the tracing kernel ----------------------------------------------------------
__global__ void __launch_bounds__(kWarps * 32)
k_trace(const Job *__restrict__ jobs, int n_jobs, TraceLaunch L) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const size_t per_warp = smem_per_warp(L);
  const uint32_t gwarp = blockIdx.x * kWarps + warp;
  WarpWork W = carve(smem + per_warp * warp, L, L.g_work ? L.g_work + (size_t)gwarp * L.g_work_words : nullptr);
  SmemStack vstk{W.stk + lane};

  uint64_t c_steps = 0, c_prim = 0, c_op = 0, c_flops = 0, c_sub = 0, c_fin = 0;
  uint32_t c_err = 0;

  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(L.item_counter, 1u);
    item = __shfl_sync(0xFFFFFFFFu, item, 0);
    if (item >= L.n_items) break;
    const int jb = find_job_tile(jobs, n_jobs, item);
    const Job &job = jobs[jb];
    const DevScene &sc = job.sc;
    const DevCamera &cam = job.cam;
    const TraceParams &tp = job.tp;
    const uint32_t tile = item - job.tile_base;
    const int T = job.tl.tile;
    const int tx = (int)(tile % (uint32_t)job.tl.tiles_x), ty = (int)(tile / (uint32_t)job.tl.tiles_x);
    const int x0 = tx * T, y0 = ty * T;
    const int tw = min(T, cam.W - x0), th = min(T, cam.H - y0);
    const int nr = tw * th;
    const uint32_t lbeg = job.tl.offsets[tile], len = job.tl.offsets[tile + 1] - lbeg;
    const float *zin_l = job.tl.z_in + lbeg;
    const float *zout_l = job.tl.z_out + lbeg;
    const uint32_t *prim_l = job.tl.prim + lbeg;

    for (int r = lane; r < nr; r += 32) {
      W.ray_z[r] = 0.f;
      W.ray_st[r] = 0u;
      W.alive[r] = (uint16_t)r;
    }
    int n_alive = nr;
    uint32_t next = 0;
    int n_act = 0, cur = 0;
    float z_end = 0.f, maxze = -INFINITY;
    __syncwarp();

    while (n_alive > 0) {
      // ---- discard active primitives with z_e <= z_end (Sec. 8) ----
      {
        int kept = 0;
        float mz = -INFINITY;
        for (int b = 0; b < n_act; b += 32) {
          const int i = b + lane;
          const bool v = i < n_act;
          const float ze = v ? W.act_ze[cur][i] : -INFINITY;
          const uint32_t ad = v ? W.act[cur][i] : 0u;
          const bool keep = v && ze > z_end;
          const uint32_t km = __ballot_sync(0xFFFFFFFFu, keep);
          if (keep) {
            const int dst = kept + __popc(km & lanemask_lt());
            W.act[cur ^ 1][dst] = ad;
            W.act_ze[cur ^ 1][dst] = ze;
            mz = fmaxf(mz, ze);
          }
          kept += __popc(km);
        }
        n_act = kept;
        cur ^= 1;
        maxze = warp_max(mz);
        __syncwarp();
      }
      if (n_act == 0 && next >= len) break;  // no primitive left: remaining rays miss
      // ---- fetch new primitives of interest (four conditions of Sec. 8) ----
      float z_begin = z_end;
      int take = 0;
      if (next < len) {
        z_begin = fmaxf(z_end, __ldg(zin_l + next));
        const uint32_t c = next + (uint32_t)lane;
        const bool valid = lane < tp.max_new && c < len;
        const float zb = valid ? __ldg(zin_l + c) : INFINITY;
        const float ze = valid ? __ldg(zout_l + c) : -INFINITY;
        const uint32_t pa = valid ? __ldg(prim_l + c) : 0xFFFFFFFFu;
        // exclusive running max of exit depths (including the active set)
        float run = ze;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          float y = __shfl_up_sync(0xFFFFFFFFu, run, o);
          if (lane >= o) run = fmaxf(run, y);
        }
        float excl = __shfl_up_sync(0xFFFFFFFFu, run, 1);
        excl = lane == 0 ? maxze : fmaxf(excl, maxze);
        const bool ok = valid && ((lane == 0 && n_act == 0) ||
                                  (zb <= excl && zb - z_begin < tp.depth_slab));
        const uint32_t fail = __ballot_sync(0xFFFFFFFFu, !ok);
        take = fail ? __ffs(fail) - 1 : 32;
        const bool taken = lane < take;
        maxze = warp_max(taken ? fmaxf(ze, maxze) : maxze);
        // ---- sorted merge by node address (Algorithm 1 needs address order) ----
        int rank_new = 0;
        for (int j = 0; j < take; ++j) {
          const uint32_t o = __shfl_sync(0xFFFFFFFFu, pa, j);
          rank_new += (o < pa) ? 1 : 0;
        }
        const uint32_t *A = W.act[cur];
        const float *AZ = W.act_ze[cur];
        uint32_t *B = W.act[cur ^ 1];
        float *BZ = W.act_ze[cur ^ 1];
        if (taken) {
          int lo = 0, hi = n_act;  // number of active addresses < pa
          while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (A[mid] < pa) lo = mid + 1; else hi = mid;
          }
          B[rank_new + lo] = pa;
          BZ[rank_new + lo] = ze;
        }
        for (int b = 0; b < n_act; b += 32) {
          const int i = b + lane;
          uint32_t ad = i < n_act ? A[i] : 0xFFFFFFFFu;
          int before = 0;
          for (int j = 0; j < take; ++j) {
            const uint32_t o = __shfl_sync(0xFFFFFFFFu, pa, j);
            before += (o < ad) ? 1 : 0;
          }
          if (i < n_act) {
            B[i + before] = ad;
            BZ[i + before] = AZ[i];
          }
        }
        n_act += take;
        cur ^= 1;
        next += (uint32_t)take;
      }
      z_end = next < len ? fminf(__ldg(zin_l + next), maxze) : maxze;
      __syncwarp();

      // ---- pruned view (Algorithm 1), one lane ----
      ViewInfo vi;
      if (lane == 0) vi = build_view(sc, W.act[cur], n_act, W.view, W.bstk, L.stack_slots);
      vi.n_view = __shfl_sync(0xFFFFFFFFu, vi.n_view, 0);
      vi.root_used = __shfl_sync(0xFFFFFFFFu, vi.root_used, 0);
      vi.n_prim = __shfl_sync(0xFFFFFFFFu, vi.n_prim, 0);
      vi.n_op = __shfl_sync(0xFFFFFFFFu, vi.n_op, 0);
      vi.flops = __shfl_sync(0xFFFFFFFFu, vi.flops, 0);
      vi.err = __shfl_sync(0xFFFFFFFFu, vi.err, 0);
      __syncwarp();
      c_sub += 1;
      if (vi.err) { c_err |= (uint32_t)vi.err; break; }
      if (!vi.root_used) continue;  // f_A = +inf: no crossing in this subfrustum

      // ---- synchronized sphere tracing of [z_begin, z_end] with ray refill ----
      int head = 0;
      int ray = -1;
      float z = 0.f, dx = 0.f, dy = 0.f, dz = 0.f, inv_ld = 0.f;
      uint32_t steps = 0;
      uint32_t live_steps = 0;
      int n_hits = 0;
      const float eps = tp.eps;
      for (;;) {
        const uint32_t need = __ballot_sync(0xFFFFFFFFu, ray < 0);
        if (need && head < n_alive) {
          const int rk = __popc(need & lanemask_lt());
          if (ray < 0 && head + rk < n_alive) {
            ray = W.alive[head + rk];
            z = fmaxf(W.ray_z[ray], z_begin);
            steps = W.ray_st[ray] & 0xFFFFFFu;
            float d[3];
            pixel_ray(cam, x0 + ray % tw, y0 + ray / tw, d);
            dx = d[0]; dy = d[1]; dz = d[2];
            inv_ld = 1.0f / (tp.lipschitz * sqrtf(dx * dx + dy * dy + dz * dz));
          }
          head = min(n_alive, head + __popc(need));
        }
        const bool live = ray >= 0;
        if (!__any_sync(0xFFFFFFFFu, live)) break;
        const float p[3] = {cam.o[0] + z * dx, cam.o[1] + z * dy, cam.o[2] + z * dz};
        const float f = eval_view<float>(W.view, vi.n_view, sc.rec, p, vstk);
        bool hit = false;
        if (live) {
          ++steps;
          ++live_steps;
          if (f <= eps) {
            hit = true;
          } else {
            z += f * inv_ld;
            if (z >= z_end) {
              W.ray_z[ray] = z_end;
              W.ray_st[ray] = steps;
              ray = -1;
            } else if ((int)steps >= tp.max_steps) {
              W.ray_st[ray] = steps | (R_UNCONV << 24);
              const int px = x0 + ray % tw, py = y0 + ray / tw;
              const size_t o = (size_t)py * cam.W + px;
              job.out.depth[o] = INFINITY;
              job.out.normal[3 * o] = 0.f; job.out.normal[3 * o + 1] = 0.f; job.out.normal[3 * o + 2] = 0.f;
              job.out.evals[o] = steps;
              job.out.flags[o] = 2;
              ray = -1;
            }
          }
        }
        const uint32_t hm = __ballot_sync(0xFFFFFFFFu, hit);
        if (hit) {
          W.hits[n_hits + __popc(hm & lanemask_lt())] = (uint16_t)ray;
          W.ray_z[ray] = z;
          W.ray_st[ray] = steps | (R_HIT << 24);
          ray = -1;
        }
        n_hits += __popc(hm);
      }
      c_steps += live_steps;
      c_prim += (uint64_t)live_steps * vi.n_prim;
      c_op += (uint64_t)live_steps * vi.n_op;
      c_flops += (uint64_t)live_steps * (vi.flops + kFlopsStep);
      __syncwarp();

      // ---- hit refinement: Newton on the ray, normal = grad f_A ----
      for (int b = 0; b < n_hits; b += 32) {
        const int idx = b + lane;
        const bool v = idx < n_hits;
        const int r = v ? W.hits[idx] : 0;
        float zz = v ? W.ray_z[r] : z_begin;
        float d[3];
        pixel_ray(cam, x0 + r % tw, y0 + r / tw, d);
        const float dn = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const float lim = tp.newton_clamp / dn;
        bool beyond = false;  // the crossing lies past z_end: not this subfrustum's
        for (int it = 0; it < tp.newton_iters; ++it) {
          Dual<1> pd[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) { pd[k].v = cam.o[k] + zz * d[k]; pd[k].g[0] = d[k]; }
          LocalStack<Dual<1>> ls;
          const Dual<1> fd = eval_view<Dual<1>>(W.view, vi.n_view, sc.rec, pd, ls);
          beyond = false;
          if (fd.g[0] != 0.f && isfinite(fd.v)) {
            float step = -fd.v / fd.g[0];
            step = fminf(fmaxf(step, -lim), lim);
            beyond = zz + step > z_end && fd.v > 0.f;
            zz = fminf(fmaxf(zz + step, z_begin), z_end);
          }
        }
        Dual<3> pg[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          pg[k].v = cam.o[k] + zz * d[k];
          pg[k].g[0] = k == 0 ? 1.f : 0.f;
          pg[k].g[1] = k == 1 ? 1.f : 0.f;
          pg[k].g[2] = k == 2 ? 1.f : 0.f;
        }
        LocalStack<Dual<3>> ls3;
        const Dual<3> fg = eval_view<Dual<3>>(W.view, vi.n_view, sc.rec, pg, ls3);
        if (v && beyond) {
          // Hand the ray back: the next subfrustum starts at z_end and owns
          // the crossing.
          W.ray_z[r] = z_end;
          W.ray_st[r] = W.ray_st[r] & 0xFFFFFFu;
        } else if (v) {
          const float gn = sqrtf(fg.g[0] * fg.g[0] + fg.g[1] * fg.g[1] + fg.g[2] * fg.g[2]);
          const float ig = gn > 0.f ? 1.f / gn : 0.f;
          const int px = x0 + r % tw, py = y0 + r / tw;
          const size_t o = (size_t)py * cam.W + px;
          job.out.depth[o] = zz * dn;
          job.out.normal[3 * o] = fg.g[0] * ig;
          job.out.normal[3 * o + 1] = fg.g[1] * ig;
          job.out.normal[3 * o + 2] = fg.g[2] * ig;
          job.out.evals[o] = W.ray_st[r] & 0xFFFFFFu;
          job.out.flags[o] = 1;
          c_fin += (uint64_t)tp.newton_iters + 1;
        }
      }
      __syncwarp();

      // ---- drop finished rays from the pending list ----
      {
        int kept = 0;
        for (int b = 0; b < n_alive; b += 32) {
          const int i = b + lane;
          const int r = i < n_alive ? W.alive[i] : 0;
          const bool keep = i < n_alive && (W.ray_st[r] >> 24) == R_ALIVE;
          const uint32_t km = __ballot_sync(0xFFFFFFFFu, keep);
          __syncwarp();
          if (keep) W.alive[kept + __popc(km & lanemask_lt())] = (uint16_t)r;
          kept += __popc(km);
          __syncwarp();
        }
        n_alive = kept;
      }
    }
    // ---- rays still pending when the list is exhausted: misses ----
    for (int i = lane; i < n_alive; i += 32) {
      const int r = W.alive[i];
      const int px = x0 + r % tw, py = y0 + r / tw;
      const size_t o = (size_t)py * cam.W + px;
      job.out.depth[o] = INFINITY;
      job.out.normal[3 * o] = 0.f; job.out.normal[3 * o + 1] = 0.f; job.out.normal[3 * o + 2] = 0.f;
      job.out.evals[o] = W.ray_st[r] & 0xFFFFFFu;
      job.out.flags[o] = 0;
    }
    __syncwarp();
  }

  if (L.counters) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      c_steps += __shfl_xor_sync(0xFFFFFFFFu, c_steps, o);
      c_prim += __shfl_xor_sync(0xFFFFFFFFu, c_prim, o);
      c_op += __shfl_xor_sync(0xFFFFFFFFu, c_op, o);
      c_flops += __shfl_xor_sync(0xFFFFFFFFu, c_flops, o);
      c_fin += __shfl_xor_sync(0xFFFFFFFFu, c_fin, o);
    }
    if (lane == 0) {
      atomicAdd((unsigned long long *)&L.counters[0], (unsigned long long)c_steps);
      atomicAdd((unsigned long long *)&L.counters[1], (unsigned long long)c_prim);
      atomicAdd((unsigned long long *)&L.counters[2], (unsigned long long)c_op);
      atomicAdd((unsigned long long *)&L.counters[3], (unsigned long long)c_flops);
      atomicAdd((unsigned long long *)&L.counters[4], (unsigned long long)c_sub);
      atomicAdd((unsigned long long *)&L.counters[6], (unsigned long long)c_fin);
      if (c_err) atomicOr((unsigned long long *)&L.counters[7], (unsigned long long)c_err);
    }
  }
}

// ---- inspection kernels: the same view build and evaluator as k_trace ----------
__global__ void k_pruned_view(DevScene sc, const uint32_t *act, int n, uint32_t *view, uint32_t *vaddr,
                              int32_t *info, uint32_t *bstk, int stack_cap) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ViewInfo vi = build_view(sc, act, n, view, bstk, stack_cap, vaddr);
  info[0] = vi.n_view;
  info[1] = vi.root_used;
  info[2] = vi.err;
  info[3] = vi.n_prim;
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
    f[i] = eval_view<float>(view, n_view, sc.rec, p, ls);
  } else {
    Dual<3> p[3];
    for (int k = 0; k < 3; ++k) {
      p[k].v = pts[3 * i + k];
      p[k].g[0] = k == 0; p[k].g[1] = k == 1; p[k].g[2] = k == 2;
    }
    LocalStack<Dual<3>> ls;
    Dual<3> r = eval_view<Dual<3>>(view, n_view, sc.rec, p, ls);
    f[i] = r.v;
    grad[3 * i] = r.g[0]; grad[3 * i + 1] = r.g[1]; grad[3 * i + 2] = r.g[2];
  }
}

void launch_pruned_view(const DevScene &sc, const uint32_t *act, int n, uint32_t *view, uint32_t *vaddr,
                        int32_t *info, uint32_t *bstk, int stack_cap, cudaStream_t s) {
  count_launch(), k_pruned_view<<<1, 32, 0, s>>>(sc, act, n, view, vaddr, info, bstk, stack_cap);
}

void launch_eval_view(const DevScene &sc, const uint32_t *view, const int32_t *info, const float *pts, int npts,
                      float *f, float *grad, cudaStream_t s) {
  if (npts > 0) count_launch(), k_eval_view<<<(npts + 127) / 128, 128, 0, s>>>(sc, view, info, pts, npts, f, grad);
}

cudaError_t trace_launch(const Job *jobs, int n_jobs, const TraceLaunch &L, int n_sm, cudaStream_t s) {
  const size_t smem = trace_smem_per_warp(L) * kWarps;
  cudaError_t e = cudaFuncSetAttribute(k_trace, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace, kWarps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  count_launch(), k_trace<<<n_sm * per_sm, kWarps * 32, smem, s>>>(jobs, n_jobs, L);
  return cudaGetLastError();
}

int trace_ctas_per_sm(const TraceLaunch &L) {
  const size_t smem = trace_smem_per_warp(L) * kWarps;
  if (cudaFuncSetAttribute(k_trace, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace, kWarps * 32, smem);
  return per_sm;
}

}  // namespace st
