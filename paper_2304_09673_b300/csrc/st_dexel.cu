// st_dexel.cu -- the non-synchronized variants the paper compares its
// pipeline against (Table 1, "ParentPtr/Full" and "FastPtr/Full"): a
// full-resolution A-buffer (one list of primitive fragments per pixel, a
// "dexel" buffer) and per-pixel sphere tracing in which every field
// evaluation runs the sparse bottom-up traversal of Algorithm 1 directly on
// the ray's own active primitives, with parent pointers (Sec. 7.1) or fast
// ancestor pointers (Sec. 7.2), instead of evaluating a pruned view shared by
// a tile.
//
//   k_dexel_pass   one CTA per screen tile, one thread per pixel: the pixel's
//                  centre ray against the volumes of interest of the tile's
//                  A-buffer list (staged in shared memory), with the FP32
//                  test of the tile culling; counts per pixel, then (second
//                  pass) writes (z_in, address) keys and z_out into the
//                  pixel's CSR segment.  A tile list holds every primitive
//                  hit by a ray of the tile, so the pixel lists equal
//                  brute-force per-pixel culling.
//   k_seg_sort_small  insertion sort of segments of at most 32 entries, one
//                  thread each (longer ones use the tile sort);
//   k_trace_dexel  one thread per pixel ray (persistent grid, 8x4 pixel
//                  blocks per warp): the ray's own list is cut into
//                  subintervals by the rule of Sec. 8 (discard, fetch up to
//                  max_new with no empty space and within the depth slab,
//                  z_end = min(next entry, last exit)), as st_trace does per
//                  tile; plain sphere tracing with f_A from eval_sparse,
//                  steps clamped at z_end, Newton refinement and the
//                  gradient normal as in st_trace.
#include <cstdint>

#include "st_field.cuh"
#include "st_geom.cuh"
#include "st_kernels.h"

namespace st {

namespace {

constexpr int kDexelChunk = 64;   // tile-list entries staged per round

// One thread per pixel of a tile: up to 32 x 32 = 1024 threads.
template <bool kFill>
__global__ void __launch_bounds__(1024) k_dexel_pass(Job job, uint32_t *count, const uint32_t *pix_off, uint64_t *keys,
                                                     float *zo_tmp) {
  __shared__ Voi s_v[kDexelChunk];
  __shared__ VoiRay s_q[kDexelChunk];
  const DevCamera &cam = job.cam;
  const int T = job.tl.tile;
  const uint32_t n_tiles = (uint32_t)job.tl.tiles_x * (uint32_t)job.tl.tiles_y;
  for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int tx = (int)(t % (uint32_t)job.tl.tiles_x), ty = (int)(t / (uint32_t)job.tl.tiles_x);
    const int px = tx * T + (int)threadIdx.x % T, py = ty * T + (int)threadIdx.x / T;
    const bool valid = px < cam.W && py < cam.H;
    const uint32_t pix = valid ? (uint32_t)py * (uint32_t)cam.W + (uint32_t)px : 0u;
    float d[3];
    pixel_ray(cam, valid ? px : 0, valid ? py : 0, d);
    const uint32_t beg = job.tl.offsets[t], end = job.tl.offsets[t + 1];
    uint32_t n = 0, dst = 0;
    if (kFill && valid) dst = pix_off[pix];
    for (uint32_t c = beg; c < end; c += kDexelChunk) {
      const uint32_t m = min((uint32_t)kDexelChunk, end - c);
      __syncthreads();
      if (threadIdx.x < m) {
        const uint32_t a = job.tl.prim[c + threadIdx.x];
        load_voi(job.sc, job.sc.prim_index[a], s_v[threadIdx.x], s_q[threadIdx.x].cc.wa);
        voi_ray_setup(s_v[threadIdx.x], cam, s_q[threadIdx.x]);
      }
      __syncthreads();
      if (!valid) continue;
      for (uint32_t k = 0; k < m; ++k) {
        float t0, t1;
        if (!voi_ray_hit(s_v[k], s_q[k], d, t0, t1)) continue;
        if (kFill) {
          keys[dst + n] = ((uint64_t)__float_as_uint(t0) << 32) | (uint64_t)job.tl.prim[c + k];
          zo_tmp[dst + n] = t1;
        }
        ++n;
      }
    }
    if (!kFill && valid) count[pix] = n;
  }
}

// Segments of 2..32 entries: insertion sort by key, one thread per segment.
__global__ void k_seg_sort_small(const uint32_t *offsets, uint32_t n_segs, const uint64_t *keys,
                                 const float *z_out_in, float *z_in, float *z_out, uint32_t *prim) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n_segs; t += gridDim.x * blockDim.x) {
    const uint32_t beg = offsets[t], len = offsets[t + 1] - beg;
    if (len < 2 || len > 32) continue;
    uint64_t k[32];
    float v[32];
    for (uint32_t i = 0; i < len; ++i) {
      const uint64_t key = keys[beg + i];
      const float val = z_out_in[beg + i];
      uint32_t j = i;
      while (j > 0 && k[j - 1] > key) { k[j] = k[j - 1]; v[j] = v[j - 1]; --j; }
      k[j] = key;
      v[j] = val;
    }
    for (uint32_t i = 0; i < len; ++i) {
      z_in[beg + i] = __uint_as_float((uint32_t)(k[i] >> 32));
      prim[beg + i] = (uint32_t)k[i];
      z_out[beg + i] = v[i];
    }
  }
}

// ---- Algorithm 1 with field values -----------------------------------------
// Active primitive i of a traversal: its post-order address.
struct ActDexel {   // a ray's active set in the strided scratch (address, z_out bits)
  const uint2 *a;
  uint32_t stride;
  __device__ __forceinline__ uint32_t operator()(int i) const { return a[(size_t)i * stride].x; }
};
struct ActPlain {
  const uint32_t *a;
  __device__ __forceinline__ uint32_t operator()(int i) const { return a[i]; }
};

struct SparseCount {
  uint32_t visits = 0;   // operators reached by the climbs (both pointer kinds)
  uint32_t ops = 0;      // operators evaluated (both operands used)
  uint32_t err = 0;      // ST_STATUS_* bits
};

template <class T>
__device__ __forceinline__ T prim_value(const DevScene &sc, uint32_t a, uint32_t kind, const T p[3]) {
  const float4 *q = sc.rec + __ldg(sc.rec_off + a);
  switch (kind) {
    case ST_PRIM_SPHERE: return sd_sphere<T>(q[0], p);
    case ST_PRIM_RBOX: return sd_rbox<T>(q[0], q[1], q[2], q[3], p);
    case ST_PRIM_CAPSULE: return sd_capsule<T>(q[0], q[2], p);
    default: return sd_further<T>(prim_view_code(kind), q, p[0], p[1], p[2]);
  }
}

template <class T>
__device__ __forceinline__ T op_value(const DevScene &sc, uint32_t a, uint32_t kind, const T &l, const T &r) {
  const uint32_t code = kind - ST_OP_UNION + V_UNION;
  if (code <= V_DIFF) return op_compact_any<T>(code, sc.rec[__ldg(sc.rec_off + a)], l, r);
  return op_sharp_any<T>(code, l, r);
}

// The traversal stacks one branch per ancestor reached through a right edge
// whose left subtree holds an active primitive, so it never holds more
// entries than Algorithm 3's post-order stack, which scene creation bounds
// by ST_MAX_STACK.
constexpr int kSparseStack = ST_MAX_STACK + 2;

// f_A at p by Algorithm 1 with TYPE = field value (direct evaluation): the
// active primitives are taken in address order; from each one the traversal
// climbs ancestor pointers until the shadowing condition (the ancestor lies
// after the next active primitive) or the root, evaluating on the way every
// operator whose two operands are both present (the left one on top of the
// stack), and stacks the branch otherwise.  kFast: fast ancestor pointers,
// the ancestor clamped by the one stacked on top, popRequiredA or
// popRequiredB (Sec. 7.2); else parent pointers and popRequiredA (Sec. 7.1).
// A lone operand passes through an operator or is blocked according to the
// operator's ignore bits, and an operator with a blocked operand takes the
// other operand, or +inf when none is used (the usage rule of Sec. 9), so
// the value equals Algorithm 3 over the pruned view of the same set.
template <bool kFast, class T, class Act>
__device__ __forceinline__ T eval_sparse(const DevScene &sc, const Act &act, int n, const T p[3], SparseCount &cnt) {
  uint32_t bw[kSparseStack];   // ancestor | usage << 31
  T bv[kSparseStack];
  int sp = 0;
  constexpr uint32_t NO = 0x7FFFFFFFu;   // no ancestor: above every address
  auto anc_of = [&](uint32_t a, uint32_t blob) -> uint32_t {
    if (kFast) {
      const uint32_t x = blob_anc(blob);
      return x == kNoAnc ? NO : x;
    }
    const uint32_t x = __ldg(sc.lift + a);
    return x == 0xFFFFFFFFu ? NO : x;
  };
  for (int i = 0; i < n; ++i) {
    const uint32_t P = act(i);
    uint32_t nb = __ldg(sc.blob + P);
    uint32_t anc = anc_of(P, nb);
    uint32_t u = 1, isl = blob_isleft(nb);
    T val = prim_value<T>(sc, P, blob_kind(nb), p);
    if (kFast && sp > 0) anc = min(anc, bw[sp - 1] & NO);
    const uint32_t next = i + 1 < n ? act(i + 1) : 0u;
    for (int guard = 0;; ++guard) {
      if (i + 1 < n) {
        if (anc > next) break;
      } else if (sp == 0 && anc == NO) {
        break;
      }
      if (anc >= (uint32_t)sc.n_nodes || guard > sc.n_nodes) { cnt.err |= ST_STATUS_VIEW; return T(INFINITY); }
      const uint32_t op = anc;
      const uint32_t ab = __ldg(sc.blob + op);
      const uint32_t a_anc = anc_of(op, ab);
      const uint32_t m = blob_igm(ab);
      ++cnt.visits;
      bool popped = false;
      if (sp > 0) {
        const uint32_t c = bw[sp - 1], c_anc = c & NO;
        bool req = op == c_anc;                                              // popRequiredA
        if (kFast) req = req || (a_anc >= c_anc && (a_anc == NO || blob_isleft(ab)));  // popRequiredB
        if (req) {
          const uint32_t b = ((c >> 31) << 1) | u;
          --sp;
          const bool ok = ((~b) & m & 3u) == 0u;
          if (ok && b == 3u) {
            val = op_value<T>(sc, op, blob_kind(ab), bv[sp], val);
            ++cnt.ops;
          } else if (!ok || b == 0u) {
            val = T(INFINITY);
          } else if (b == 2u) {
            val = bv[sp];   // only the left operand is used
          }
          u = (ok && b != 0u) ? 1u : 0u;
          popped = true;
        }
      }
      if (!popped) {
        const uint32_t b = isl ? (u << 1) : u;
        const bool ok = ((~b) & m & 3u) == 0u;
        u = (ok && b != 0u) ? 1u : 0u;
      }
      nb = ab;
      isl = blob_isleft(ab);
      anc = a_anc;
      if (kFast && sp > 0) anc = min(anc, bw[sp - 1] & NO);
    }
    if (sp >= kSparseStack) { cnt.err |= ST_STATUS_STACK; return T(INFINITY); }
    bw[sp] = anc | (u << 31);
    bv[sp] = val;
    ++sp;
  }
  if (sp != 1) { cnt.err |= ST_STATUS_VIEW; return T(INFINITY); }
  return (bw[0] >> 31) ? bv[0] : T(INFINITY);
}

template <bool kFast>
__global__ void k_eval_sparse(DevScene sc, const uint32_t *act, int n, const float *pts, int npts, float *f,
                              uint32_t *status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npts) return;
  const float p[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
  SparseCount cnt;
  f[i] = eval_sparse<kFast, float>(sc, ActPlain{act}, n, p, cnt);
  if (cnt.err) atomicOr(status, cnt.err);
}

// ---- per-pixel tracing ---------------------------------------------------------
template <bool kFast>
__global__ void __launch_bounds__(128) k_trace_dexel(Job job, DexelLaunch D) {
  const DevCamera &cam = job.cam;
  const DevScene &sc = job.sc;
  const TraceParams &tp = job.tp;
  const int lane = threadIdx.x & 31;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t bx_n = ((uint32_t)cam.W + 7u) / 8u, by_n = ((uint32_t)cam.H + 3u) / 4u;
  const uint32_t n_items = bx_n * by_n * 32u;
  const float eps = tp.eps, L = tp.lipschitz;
  uint64_t c_steps = 0, c_prim = 0, c_visit = 0, c_ops = 0, c_int = 0;
  uint32_t c_err = 0;
  const ActDexel act{D.act + tid, D.n_threads};
  uint2 *const slot = D.act + tid;
  const size_t stride = D.n_threads;
  for (;;) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(D.pixel_counter, 32u);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (base >= n_items) break;
    const uint32_t k = base + (uint32_t)lane, blk = k / 32u, in = k % 32u;
    const int px = (int)((blk % bx_n) * 8u + in % 8u), py = (int)((blk / bx_n) * 4u + in / 8u);
    if (px >= cam.W || py >= cam.H) continue;
    const size_t o = (size_t)py * cam.W + px;
    float d[3];
    pixel_ray(cam, px, py, d);
    const float dn = sqrtf(fma_(d[0], d[0], fma_(d[1], d[1], mul_(d[2], d[2]))));
    const float inv_ld = 1.0f / mul_(L, dn);
    const float lim = tp.newton_clamp / dn;
    const uint32_t beg = D.offsets[o], end = D.offsets[o + 1];
    uint32_t nxt = beg, steps = 0;
    int n_act = 0;
    int result = 0;   // 0 miss, 1 hit, 2 step cap
    float z = kZNear, zend = 0.f, zz = 0.f, g[3] = {0.f, 0.f, 0.f};
    while (result == 0) {
      // The subinterval rule of Sec. 8 on the ray's own list: drop fragments
      // that end at or before the previous end, then fetch (up to max_new
      // new ones, no empty space, within the depth slab), active set in
      // address order.
      int w = 0;
      float maxze = -INFINITY;
      for (int i = 0; i < n_act; ++i) {
        const uint2 e = slot[(size_t)i * stride];
        const float zo = __uint_as_float(e.y);
        if (zo > zend) {
          slot[(size_t)w++ * stride] = e;
          maxze = fmaxf(maxze, zo);
        }
      }
      n_act = w;
      if (n_act == 0 && nxt >= end) break;   // past the last fragment: miss
      float zb = zend;
      if (nxt < end) {
        zb = fmaxf(zend, D.z_in[nxt]);
        const int n0 = n_act;
        float run = maxze;
        int take = 0;
        for (uint32_t c = nxt; c < end && take < tp.max_new; ++c) {
          const float zi = D.z_in[c], zo = D.z_out[c];
          const bool ok = (take == 0 && n0 == 0) || (zi <= run && zi - zb < tp.depth_slab);
          if (!ok) break;
          const uint2 e = make_uint2(D.prim[c], __float_as_uint(zo));
          int j = n_act;
          while (j > 0 && slot[(size_t)(j - 1) * stride].x > e.x) {
            slot[(size_t)j * stride] = slot[(size_t)(j - 1) * stride];
            --j;
          }
          slot[(size_t)j * stride] = e;
          ++n_act;
          run = fmaxf(run, zo);
          ++take;
        }
        maxze = run;
        nxt += (uint32_t)take;
      }
      zend = nxt < end ? fminf(D.z_in[nxt], maxze) : maxze;
      z = fmaxf(z, zb);
      if (!(z < zend)) continue;
      ++c_int;
      const float z_b = zb, z_end = zend;
      bool hit = false;
      for (;;) {
        const float p[3] = {fma_(z, d[0], cam.o[0]), fma_(z, d[1], cam.o[1]), fma_(z, d[2], cam.o[2])};
        SparseCount cnt;
        const float f = eval_sparse<kFast, float>(sc, act, n_act, p, cnt);
        c_visit += cnt.visits;
        c_ops += cnt.ops;
        c_err |= cnt.err;
        ++steps;
        ++c_steps;
        c_prim += (uint64_t)n_act;
        if (f <= eps) { hit = true; break; }
        if ((int)steps >= tp.max_steps) { result = 2; break; }
        z = add_(z, mul_(fabsf(f), inv_ld));
        // f_A has the sign of f only inside the subinterval: a step never
        // goes past its end (f_A is +inf where A's branch is blocked).
        if (z >= z_end) { z = z_end; break; }
      }
      if (!hit) continue;
      // Newton along the ray on f_A, then the gradient from three axis
      // derivatives (as st_trace's hit refinement); a crossing beyond z_end
      // returns the ray to marching from z_end.
      zz = z;
      bool beyond = false, done = false;
      for (int it = 0; it < tp.newton_iters && !done; ++it) {
        Dual<1> pd[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) { pd[j].v = cam.o[j] + zz * d[j]; pd[j].g[0] = d[j]; }
        SparseCount cnt;
        const Dual<1> fd = eval_sparse<kFast, Dual<1>>(sc, act, n_act, pd, cnt);
        c_err |= cnt.err;
        // a first sample inside the solid at the near plane: clipped hit
        if (it == 0 && zz <= kZNear && fd.v < -eps) break;
        beyond = false;
        if (fd.g[0] != 0.f && isfinite(fd.v)) {
          float step = -fd.v / fd.g[0];
          step = fminf(fmaxf(step, -lim), lim);
          beyond = zz + step > z_end && fd.v > 0.f;
          const float zn = fminf(fmaxf(zz + step, z_b), z_end);
          if (fabsf(zn - zz) <= 1e-6f * zz) done = true;
          zz = zn;
        } else {
          done = true;
        }
      }
      if (beyond) {
        z = z_end;
        continue;
      }
      for (int ax = 0; ax < 3; ++ax) {
        Dual<1> pd[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) { pd[j].v = cam.o[j] + zz * d[j]; pd[j].g[0] = j == ax ? 1.f : 0.f; }
        SparseCount cnt;
        g[ax] = eval_sparse<kFast, Dual<1>>(sc, act, n_act, pd, cnt).g[0];
        c_err |= cnt.err;
      }
      result = 1;
    }
    DevOut &out = job.out;
    if (result == 1) {
      const float gn = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
      const float ig = gn > 0.f ? 1.f / gn : 0.f;
      out.depth[o] = zz * dn;
      out.normal[3 * o] = g[0] * ig;
      out.normal[3 * o + 1] = g[1] * ig;
      out.normal[3 * o + 2] = g[2] * ig;
      out.flags[o] = 1;
    } else {
      out.depth[o] = INFINITY;
      out.normal[3 * o] = 0.f;
      out.normal[3 * o + 1] = 0.f;
      out.normal[3 * o + 2] = 0.f;
      out.flags[o] = result == 2 ? 2 : 0;
    }
    out.evals[o] = steps;
  }
  if (D.counters) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      c_steps += __shfl_xor_sync(0xFFFFFFFFu, c_steps, s);
      c_prim += __shfl_xor_sync(0xFFFFFFFFu, c_prim, s);
      c_visit += __shfl_xor_sync(0xFFFFFFFFu, c_visit, s);
      c_ops += __shfl_xor_sync(0xFFFFFFFFu, c_ops, s);
      c_int += __shfl_xor_sync(0xFFFFFFFFu, c_int, s);
      c_err |= __shfl_xor_sync(0xFFFFFFFFu, c_err, s);
    }
    if (lane == 0) {
      atomicAdd((unsigned long long *)&D.counters[0], (unsigned long long)c_steps);
      atomicAdd((unsigned long long *)&D.counters[1], (unsigned long long)c_prim);
      atomicAdd((unsigned long long *)&D.counters[2], (unsigned long long)c_visit);
      atomicAdd((unsigned long long *)&D.counters[3], (unsigned long long)c_ops);
      atomicAdd((unsigned long long *)&D.counters[4], (unsigned long long)c_int);
      if (c_err) atomicOr((unsigned long long *)&D.counters[7], (unsigned long long)c_err);
    }
  }
}

}  // namespace

void launch_dexel_pass(const Job &job, bool fill, uint32_t *count, const uint32_t *pix_off, uint64_t *keys,
                       float *zo_tmp, cudaStream_t s) {
  const uint32_t n_tiles = (uint32_t)job.tl.tiles_x * (uint32_t)job.tl.tiles_y;
  if (!n_tiles) return;
  const int threads = job.tl.tile * job.tl.tile;
  const uint32_t grid = n_tiles < 65535u ? n_tiles : 65535u;
  if (fill) count_launch(), k_dexel_pass<true><<<grid, threads, 0, s>>>(job, count, pix_off, keys, zo_tmp);
  else count_launch(), k_dexel_pass<false><<<grid, threads, 0, s>>>(job, count, pix_off, keys, zo_tmp);
}

void launch_segment_sort(const uint32_t *offsets, uint32_t n_segs, uint32_t max_len, const uint64_t *keys,
                         const float *z_out_tmp, float *z_in, float *z_out, uint32_t *prim, int n_sm, cudaStream_t s) {
  if (!n_segs) return;
  launch_copy_short(offsets, n_segs, keys, z_out_tmp, z_in, z_out, prim, s);
  if (max_len > 1)
    count_launch(), k_seg_sort_small<<<n_sm * 16, 128, 0, s>>>(offsets, n_segs, keys, z_out_tmp, z_in, z_out, prim);
  if (max_len > 32) launch_tile_sort_range(offsets, n_segs, max_len, 32, keys, z_out_tmp, z_in, z_out, prim, n_sm, s);
}

cudaError_t launch_eval_sparse(const DevScene &sc, const uint32_t *act, int n, const float *pts, int npts,
                               int fast, float *f, uint32_t *status, cudaStream_t s) {
  if (npts <= 0) return cudaSuccess;
  const int blocks = (npts + 127) / 128;
  if (fast) count_launch(), k_eval_sparse<true><<<blocks, 128, 0, s>>>(sc, act, n, pts, npts, f, status);
  else count_launch(), k_eval_sparse<false><<<blocks, 128, 0, s>>>(sc, act, n, pts, npts, f, status);
  return cudaGetLastError();
}

cudaError_t dexel_trace_grid(int fast, int n_sm, int *grid) {
  int per_sm = 0;
  cudaError_t e = fast ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_dexel<true>, 128, 0)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_dexel<false>, 128, 0);
  if (e != cudaSuccess) return e;
  *grid = n_sm * (per_sm > 0 ? per_sm : 1);
  return cudaSuccess;
}

cudaError_t launch_trace_dexel(const Job &job, const DexelLaunch &D, int fast, int grid, cudaStream_t s) {
  if (fast) count_launch(), k_trace_dexel<true><<<grid, 128, 0, s>>>(job, D);
  else count_launch(), k_trace_dexel<false><<<grid, 128, 0, s>>>(job, D);
  return cudaGetLastError();
}

}  // namespace st
