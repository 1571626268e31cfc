// st_cull.cu -- per-tile culling of blobtree primitives into a low-resolution
// A-buffer (Sec. 6), for one or many (scene, camera) jobs at once.
//
// Pipeline (all on the caller's stream):
//   k_prim_bounds  one thread per primitive: volume of interest (Sec. 6.1:
//                  primitive bound offset by its range-of-interest bound d)
//                  -> conservative screen tile rectangle -> candidate count
//   scan           candidate offsets
//   k_cull_pairs   one warp per candidate (primitive, tile): one FP32 ray per
//                  pixel centre of the tile against the volume of interest;
//                  entry = min max(t0, 0), exit = max t1 over hitting rays
//                  (the 8x8 ray/volume tests of the paper's fragment shader,
//                  Sec. 6.2, as explicit compute); kept iff a ray hits.
//                  Survivors are appended to a pair list with CTA-aggregated
//                  atomics; each pair takes its rank inside its tile.
//   scan           tile offsets (CSR), longest list
//   k_scatter      pair -> CSR slot (offset + rank)
//   k_tile_sort    per-tile bitonic sort in shared memory by
//                  (z_in, post-order address) (sorted lists, Sec. 6.2)
//   lists longer than kSortLarge (no length cap): chunks of kSortLarge
//                  entries sorted in shared memory (k_chunk_sort), then
//                  pairwise merges of sorted runs in global memory
//                  (k_merge_pass), each element placed by a binary search
//                  in the partner run
#include <cstdint>

#include "st_geom.cuh"
#include "st_kernels.h"

namespace st {

namespace {

__device__ __forceinline__ int find_job_prim(const Job *jobs, int n_jobs, uint32_t g) {
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].prim_base <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Conservative pixel rectangle of a sphere (centre C, radius rho) in view:
// returns 0 when it is off screen or behind the eye, 2 when it straddles the
// eye plane (whole screen), 1 with the rectangle [x0, x1] x [y0, y1].
__device__ int sphere_pixel_rect(const DevCamera &cam, const float C[3], float rho, int4 &px) {
  rho = rho * 1.001f + 1e-4f;
  float w[3] = {C[0] - cam.o[0], C[1] - cam.o[1], C[2] - cam.o[2]};
  float lr = sqrtf(cam.R[0] * cam.R[0] + cam.R[1] * cam.R[1] + cam.R[2] * cam.R[2]);
  float lu = sqrtf(cam.U[0] * cam.U[0] + cam.U[1] * cam.U[1] + cam.U[2] * cam.U[2]);
  float z = w[0] * cam.F[0] + w[1] * cam.F[1] + w[2] * cam.F[2];
  float x = (w[0] * cam.R[0] + w[1] * cam.R[1] + w[2] * cam.R[2]) / lr;
  float y = (w[0] * cam.U[0] + w[1] * cam.U[1] + w[2] * cam.U[2]) / lu;
  if (z < -rho) return 0;              // behind the eye
  if (z <= rho * 1.01f) return 2;      // straddles the eye plane
  float zz = z * z - rho * rho;
  float sx = sqrtf(fmaxf(x * x + zz, 0.f)), sy = sqrtf(fmaxf(y * y + zz, 0.f));
  float mx0 = (x * z - rho * sx) / zz, mx1 = (x * z + rho * sx) / zz;
  float my0 = (y * z - rho * sy) / zz, my1 = (y * z + rho * sy) / zz;
  float u0 = mx0 / lr, u1 = mx1 / lr;   // image u in [-1, 1] across the width
  float v0 = my0 / lu, v1 = my1 / lu;   // image v in [-1, 1], +1 = top row
  // pixel i has u = (2i+1)/W - 1  ->  i = ((u + 1) W - 1) / 2
  float i0 = ((u0 + 1.f) * cam.W - 1.f) * 0.5f, i1 = ((u1 + 1.f) * cam.W - 1.f) * 0.5f;
  float j0 = ((1.f - v1) * cam.H - 1.f) * 0.5f, j1 = ((1.f - v0) * cam.H - 1.f) * 0.5f;
  float fi0 = floorf(i0) - 1.f, fi1 = ceilf(i1) + 1.f;
  float fj0 = floorf(j0) - 1.f, fj1 = ceilf(j1) + 1.f;
  if (fi1 < 0.f || fj1 < 0.f || fi0 > (float)(cam.W - 1) || fj0 > (float)(cam.H - 1)) return 0;
  px.x = fi0 < 0.f ? 0 : (int)fi0;
  px.y = fj0 < 0.f ? 0 : (int)fj0;
  px.z = fi1 > (float)(cam.W - 1) ? cam.W - 1 : (int)fi1;
  px.w = fj1 > (float)(cam.H - 1) ? cam.H - 1 : (int)fj1;
  return 1;
}

// Conservative pixel rectangle of the points c +- e0 a0 +- e1 a1 +- e2 a2 (a
// box's corners; its projection is their convex hull when all lie in front
// of the eye): 0 off screen, 2 unusable (a corner near or behind the eye
// plane), 1 with the rectangle.
__device__ int box_pixel_rect(const DevCamera &cam, const Voi &v, int4 &px) {
  const float lr2 = cam.R[0] * cam.R[0] + cam.R[1] * cam.R[1] + cam.R[2] * cam.R[2];
  const float lu2 = cam.U[0] * cam.U[0] + cam.U[1] * cam.U[1] + cam.U[2] * cam.U[2];
  float imin = INFINITY, imax = -INFINITY, jmin = INFINITY, jmax = -INFINITY;
  for (int k = 0; k < 8; ++k) {
    float w[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      w[q] = v.c[q] - cam.o[q];
#pragma unroll
      for (int i = 0; i < 3; ++i) w[q] += ((k >> i) & 1 ? v.e[i] : -v.e[i]) * v.M[3 * i + q];
    }
    const float z = w[0] * cam.F[0] + w[1] * cam.F[1] + w[2] * cam.F[2];
    if (!(z > 1e-3f)) return 2;
    const float u = (w[0] * cam.R[0] + w[1] * cam.R[1] + w[2] * cam.R[2]) / (lr2 * z);
    const float vv = (w[0] * cam.U[0] + w[1] * cam.U[1] + w[2] * cam.U[2]) / (lu2 * z);
    const float i = ((u + 1.f) * cam.W - 1.f) * 0.5f, j = ((1.f - vv) * cam.H - 1.f) * 0.5f;
    imin = fminf(imin, i); imax = fmaxf(imax, i);
    jmin = fminf(jmin, j); jmax = fmaxf(jmax, j);
  }
  // one pixel plus a relative margin for rounding
  const float mi = 1.f + 1e-4f * (fabsf(imin) + fabsf(imax)), mj = 1.f + 1e-4f * (fabsf(jmin) + fabsf(jmax));
  const float fi0 = floorf(imin - mi), fi1 = ceilf(imax + mi), fj0 = floorf(jmin - mj), fj1 = ceilf(jmax + mj);
  if (fi1 < 0.f || fj1 < 0.f || fi0 > (float)(cam.W - 1) || fj0 > (float)(cam.H - 1)) return 0;
  px.x = fi0 < 0.f ? 0 : (int)fi0;
  px.y = fj0 < 0.f ? 0 : (int)fj0;
  px.z = fi1 > (float)(cam.W - 1) ? cam.W - 1 : (int)fi1;
  px.w = fj1 > (float)(cam.H - 1) ? cam.H - 1 : (int)fj1;
  return 1;
}

}  // namespace

__global__ void k_prim_bounds(const Job *jobs, int n_jobs, uint32_t n_prims_total,
                              uint32_t *cand_count, int4 *rects) {
  uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_prims_total) return;
  int jb = find_job_prim(jobs, n_jobs, g);
  const Job &job = jobs[jb];
  uint32_t j = g - job.prim_base;
  Voi v;
  load_voi(job.sc, j, v);
  // Pixel rectangle of the volume of interest: its own projection where it
  // is cheap (box corners; capsule and cylinder as the union of their end
  // spheres), else that of a bounding sphere.
  const DevCamera &cam = job.cam;
  int4 px = make_int4(0, 0, cam.W - 1, cam.H - 1);
  int st;
  if (v.fam == VOI_SPHERE) {
    st = sphere_pixel_rect(cam, v.c, v.r, px);
  } else if (v.fam == VOI_STRI) {
    // bounding sphere: the vertices' centroid, the farthest vertex + r
    const float C[3] = {(v.c[0] + v.b[0] + v.e[0]) / 3.f, (v.c[1] + v.b[1] + v.e[1]) / 3.f,
                        (v.c[2] + v.b[2] + v.e[2]) / 3.f};
    float rho = 0.f;
    for (int k = 0; k < 3; ++k) {
      const float *p = k == 0 ? v.c : (k == 1 ? v.b : v.e);
      const float dx = p[0] - C[0], dy = p[1] - C[1], dz = p[2] - C[2];
      rho = fmaxf(rho, sqrtf(dx * dx + dy * dy + dz * dz));
    }
    st = sphere_pixel_rect(cam, C, rho * 1.0001f + v.r, px);
  } else if (v.fam == VOI_BOX) {
    st = box_pixel_rect(cam, v, px);
    if (st == 2) {
      const float rho = sqrtf(v.e[0] * v.e[0] + v.e[1] * v.e[1] + v.e[2] * v.e[2]);
      st = sphere_pixel_rect(cam, v.c, rho, px);
    }
  } else {
    int4 pa, pb;
    const int sa = sphere_pixel_rect(cam, v.c, v.r, pa), sb = sphere_pixel_rect(cam, v.b, v.r, pb);
    if (sa == 2 || sb == 2) {
      st = 2;
    } else if (sa == 0 && sb == 0) {
      // both end spheres off screen: the segment between them may still cross it
      const float h[3] = {0.5f * (v.b[0] - v.c[0]), 0.5f * (v.b[1] - v.c[1]), 0.5f * (v.b[2] - v.c[2])};
      const float C[3] = {v.c[0] + h[0], v.c[1] + h[1], v.c[2] + h[2]};
      st = sphere_pixel_rect(cam, C, sqrtf(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]) + v.r, px);
    } else {
      // the hull of the two spheres projects inside the union of their
      // rectangles extended to each other
      if (sa == 0) pa = pb;
      if (sb == 0) pb = pa;
      if (sa == 0 || sb == 0) {
        const float h[3] = {0.5f * (v.b[0] - v.c[0]), 0.5f * (v.b[1] - v.c[1]), 0.5f * (v.b[2] - v.c[2])};
        const float C[3] = {v.c[0] + h[0], v.c[1] + h[1], v.c[2] + h[2]};
        st = sphere_pixel_rect(cam, C, sqrtf(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]) + v.r, px);
      } else {
        px = make_int4(min(pa.x, pb.x), min(pa.y, pb.y), max(pa.z, pb.z), max(pa.w, pb.w));
        st = 1;
      }
    }
  }
  const int T = job.tl.tile;
  int4 rect;
  if (st == 0) rect = make_int4(1, 1, 0, 0);
  else if (st == 2) rect = make_int4(0, 0, job.tl.tiles_x - 1, job.tl.tiles_y - 1);
  else rect = make_int4(px.x / T, px.y / T, px.z / T, px.w / T);
  uint32_t n = 0;
  if (rect.z >= rect.x && rect.w >= rect.y) n = (uint32_t)(rect.z - rect.x + 1) * (uint32_t)(rect.w - rect.y + 1);
  cand_count[g] = n;
  rects[g] = rect;
}

// One warp per candidate pair, PAIRS_PER_WARP pairs per warp per round, CTA
// of 8 warps; survivors are compacted in shared memory and appended with one
// atomic per CTA round.  Four CTAs per SM (64 registers): the ray tests are
// chains of dependent IEEE operations, and the extra warps hide more of
// their latency than the few spilled registers cost (measured on B300:
// 1920x1080 culling 17-20 % faster than at 86 registers and three CTAs).
constexpr int kCullWarps = 8;
constexpr int kPairsPerWarp = 8;

// The tile's pixel-centre rays against one volume of interest: this lane's
// rays (one column, rows lane / T, lane / T + 32 / T, ...), with the same
// per-ray arithmetic as pixel_ray.  Returns the lane's (min entry, max exit)
// bits (0xFFFFFFFF, 0 when none hits).
template <bool kStri>
__device__ __forceinline__ uint2 cull_rays(const Voi &v, const VoiRay &vq, const DevCamera &cam, int T, int tx,
                                           int ty, int lane) {
  uint32_t zin_bits = 0xFFFFFFFFu, zout_bits = 0u;
  // Lane -> one pixel column (T <= 32 divides 32): its u and F + u R are
  // computed once; the rows' v come from the lanes that computed them.
  const int px = tx * T + lane % T;
  const float u = ieee_sub(ieee_div((float)(2 * px + 1), (float)cam.W), 1.0f);
  const float fu[3] = {ieee_add(cam.F[0], ieee_mul(u, cam.R[0])), ieee_add(cam.F[1], ieee_mul(u, cam.R[1])),
                       ieee_add(cam.F[2], ieee_mul(u, cam.R[2]))};
  const float v_row = ieee_sub(1.0f, ieee_div((float)(2 * (ty * T + lane % T) + 1), (float)cam.H));
  const int rows_per_pass = 32 / T;
  for (int row = lane / T; row < T; row += rows_per_pass) {
    const int py = ty * T + row;
    const float vv = __shfl_sync(0xFFFFFFFFu, v_row, row);
    if (px >= cam.W || py >= cam.H) continue;
    float d[3], t0, t1;
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = ieee_add(fu[k], ieee_mul(vv, cam.U[k]));
    if (!voi_ray_hit<kStri>(v, vq, d, t0, t1)) continue;
    // t0, t1 >= 0: float order equals unsigned bit order.
    uint32_t b0 = __float_as_uint(t0), b1 = __float_as_uint(t1);
    zin_bits = b0 < zin_bits ? b0 : zin_bits;
    zout_bits = b1 > zout_bits ? b1 : zout_bits;
  }
  return make_uint2(zin_bits, zout_bits);
}

// kStri: the launch for sphere-triangle volumes only (a second launch, made
// only for scenes with rounded triangles); the first launch skips them.
// Their long ray test would otherwise weigh on every family's registers.
template <bool kStri>
__global__ void __launch_bounds__(kCullWarps * 32, 4)
k_cull_pairs(const Job *jobs, int n_jobs, const uint32_t *cand_off, uint32_t n_prims_total,
             const uint32_t *cand_total, const int4 *rects, uint32_t *tile_count,
             Pair *pairs, uint32_t pair_cap, uint32_t *pair_counter) {
  __shared__ Pair s_pairs[kCullWarps * kPairsPerWarp];
  __shared__ uint32_t s_n, s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t total = *cand_total;
  const uint32_t per_round = kCullWarps * kPairsPerWarp;
  for (uint32_t base = blockIdx.x * per_round; base < total; base += gridDim.x * per_round) {
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    // A warp's consecutive candidates almost always share their primitive:
    // its volume of interest and ray-independent terms are kept between them.
    uint32_t g = 0xFFFFFFFFu;
    int jb = 0;
    Voi v;
    VoiRay vq;
    for (int q = 0; q < kPairsPerWarp; ++q) {
      uint32_t p = base + warp * kPairsPerWarp + q;
      if (p >= total) break;
      // candidate -> primitive: the last g with cand_off[g] <= p (binary
      // search for the warp's first candidate, then a forward scan)
      uint32_t gn;
      if (g == 0xFFFFFFFFu) {
        uint32_t lo = 0, hi = n_prims_total - 1;
        while (lo < hi) {
          uint32_t mid = (lo + hi + 1) >> 1;
          if (cand_off[mid] <= p) lo = mid; else hi = mid - 1;
        }
        gn = lo;
      } else {
        gn = g;
        while (gn + 1 < n_prims_total && cand_off[gn + 1] <= p) ++gn;
      }
      if (gn != g) {
        g = gn;
        jb = find_job_prim(jobs, n_jobs, g);
        load_voi<kStri>(jobs[jb].sc, g - jobs[jb].prim_base, v, vq.cc.wa);
        if ((v.fam == VOI_STRI) == kStri) voi_ray_setup<kStri>(v, jobs[jb].cam, vq);
      }
      const Job &job = jobs[jb];
      const uint32_t j = g - job.prim_base;
      const int4 rect = rects[g];
      const uint32_t k = p - cand_off[g];
      const uint32_t rw = (uint32_t)(rect.z - rect.x + 1);
      const int tx = rect.x + (int)(k % rw), ty = rect.y + (int)(k / rw);
      const int T = job.tl.tile;
      const DevCamera &cam = job.cam;
      if ((v.fam == VOI_STRI) != kStri) continue;
      const uint2 zb = cull_rays<kStri>(v, vq, cam, T, tx, ty, lane);
      uint32_t zin_bits = zb.x, zout_bits = zb.y;
      zin_bits = __reduce_min_sync(0xFFFFFFFFu, zin_bits);
      zout_bits = __reduce_max_sync(0xFFFFFFFFu, zout_bits);
      if (lane == 0 && zin_bits != 0xFFFFFFFFu) {
        const uint32_t tg = job.tile_base + (uint32_t)(ty * job.tl.tiles_x + tx);
        Pair pr;
        pr.tile = tg;
        pr.rank = atomicAdd(&tile_count[tg], 1u);
        pr.z_in = __uint_as_float(zin_bits);
        pr.z_out = __uint_as_float(zout_bits);
        pr.addr = job.sc.prim_addr[j];
        uint32_t slot = atomicAdd(&s_n, 1u);
        s_pairs[slot] = pr;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) s_base = s_n ? atomicAdd(pair_counter, s_n) : 0u;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < s_n; i += blockDim.x) {
      uint32_t dst = s_base + i;
      if (dst < pair_cap) pairs[dst] = s_pairs[i];
    }
    __syncthreads();
  }
}

// `abort` (optional): a status word; the kernel does nothing when its
// capacity bit is set (a batch whose buffers turned out too small).
__device__ __forceinline__ bool aborted(const uint32_t *abort) {
  return abort && (*(volatile const uint32_t *)abort & ST_STATUS_CAPACITY);
}

__global__ void k_scatter(const Pair *pairs, const uint32_t *pair_counter, uint32_t pair_cap,
                          const uint32_t *offsets, uint64_t *keys, float *z_out, const uint32_t *abort) {
  if (aborted(abort)) return;
  uint32_t n = min(*pair_counter, pair_cap);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    Pair p = pairs[i];
    uint32_t dst = offsets[p.tile] + p.rank;
    if (dst >= pair_cap) continue;
    keys[dst] = ((uint64_t)__float_as_uint(p.z_in) << 32) | (uint64_t)p.addr;
    z_out[dst] = p.z_out;
  }
}

// Capacity check of a batch's fixed buffers, after the tile scan: entries
// beyond the pair buffer, or a list longer than the planned sort / active-set
// capacity, set the capacity bit of the status word.
__global__ void k_check_capacity(const uint32_t *pair_counter, uint32_t pair_cap, const uint32_t *max_overlap,
                                 uint32_t overlap_cap, uint32_t *status) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    if (*pair_counter > pair_cap || *max_overlap > overlap_cap) atomicOr(status, ST_STATUS_CAPACITY);
  }
}

// Bitonic sort of one tile's (key, z_out) list in shared memory; lists with
// len in (min_len, max_len] only (two launches cover short and long lists).
__global__ void k_tile_sort(const uint32_t *offsets, uint32_t n_tiles, const uint64_t *keys,
                            const float *z_out_in, float *z_in, float *z_out, uint32_t *prim,
                            uint32_t min_len, uint32_t max_len, const uint32_t *abort) {
  if (aborted(abort)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t *sk = reinterpret_cast<uint64_t *>(smem_raw);
  for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const uint32_t beg = offsets[t], len = offsets[t + 1] - beg;
    if (len <= min_len || len > max_len) continue;
    uint32_t n2 = 1;
    while (n2 < len) n2 <<= 1;
    float *sv = reinterpret_cast<float *>(sk + n2);
    for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x) {
      if (i < len) { sk[i] = keys[beg + i]; sv[i] = z_out_in[beg + i]; }
      else { sk[i] = ~0ull; sv[i] = 0.f; }
    }
    __syncthreads();
    for (uint32_t k = 2; k <= n2; k <<= 1) {
      for (uint32_t jj = k >> 1; jj > 0; jj >>= 1) {
        for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x) {
          uint32_t l = i ^ jj;
          if (l > i) {
            bool up = (i & k) == 0;
            uint64_t a = sk[i], b = sk[l];
            if ((a > b) == up) {
              sk[i] = b; sk[l] = a;
              float x = sv[i]; sv[i] = sv[l]; sv[l] = x;
            }
          }
        }
        __syncthreads();
      }
    }
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
      uint64_t key = sk[i];
      z_in[beg + i] = __uint_as_float((uint32_t)(key >> 32));
      prim[beg + i] = (uint32_t)key;
      z_out[beg + i] = sv[i];
    }
    __syncthreads();
  }
}

// ---- lists longer than kSortLarge -----------------------------------------------
// Keys are unique within a list (one entry per primitive and tile), so an
// element's place in a merged run is its offset in its own run plus the
// number of keys of the partner run below it.
__global__ void k_long_lists(const uint32_t *offsets, uint32_t n_tiles, uint32_t *list, uint32_t *count,
                             const uint32_t *abort) {
  if (aborted(abort)) return;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x)
    if (offsets[t + 1] - offsets[t] > kSortLarge) list[atomicAdd(count, 1u)] = t;
}

// One CTA per chunk of kSortLarge entries of a long list: bitonic sort in
// shared memory, written back in place (sorted runs of kSortLarge).
__global__ void k_chunk_sort(const uint32_t *offsets, const uint32_t *list, const uint32_t *count, uint64_t *keys,
                             float *z_out_tmp, const uint32_t *abort) {
  if (aborted(abort)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t *sk = reinterpret_cast<uint64_t *>(smem_raw);
  float *sv = reinterpret_cast<float *>(sk + kSortLarge);
  const uint32_t n_long = *count;
  for (uint32_t li = 0; li < n_long; ++li) {
    const uint32_t t = list[li];
    const uint32_t beg = offsets[t], len = offsets[t + 1] - beg;
    const uint32_t n_chunks = (len + kSortLarge - 1) / kSortLarge;
    for (uint32_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
      const uint32_t c0 = beg + c * kSortLarge, cl = min(kSortLarge, len - c * kSortLarge);
      for (uint32_t i = threadIdx.x; i < kSortLarge; i += blockDim.x) {
        if (i < cl) { sk[i] = keys[c0 + i]; sv[i] = z_out_tmp[c0 + i]; }
        else { sk[i] = ~0ull; sv[i] = 0.f; }
      }
      __syncthreads();
      for (uint32_t k = 2; k <= kSortLarge; k <<= 1) {
        for (uint32_t jj = k >> 1; jj > 0; jj >>= 1) {
          for (uint32_t i = threadIdx.x; i < kSortLarge; i += blockDim.x) {
            const uint32_t l = i ^ jj;
            if (l > i) {
              const bool up = (i & k) == 0;
              const uint64_t a = sk[i], b = sk[l];
              if ((a > b) == up) {
                sk[i] = b; sk[l] = a;
                const float x = sv[i]; sv[i] = sv[l]; sv[l] = x;
              }
            }
          }
          __syncthreads();
        }
      }
      for (uint32_t i = threadIdx.x; i < cl; i += blockDim.x) {
        keys[c0 + i] = sk[i];
        z_out_tmp[c0 + i] = sv[i];
      }
      __syncthreads();
    }
  }
}

// Sorted runs of w entries (a list's last run may be shorter) merged in
// pairs into runs of 2w.  The two buffers: A = (64-bit keys, z_out) as the
// scatter wrote them, B = the output arrays (z_in bits = key >> 32, prim =
// low word, z_out).  kFromA: read A, write B; else read B, write A.
template <bool kFromA>
__global__ void k_merge_pass(const uint32_t *offsets, const uint32_t *list, const uint32_t *count, uint32_t w,
                             uint64_t *keys, float *z_out_tmp, float *z_in, uint32_t *prim, float *z_out,
                             const uint32_t *abort) {
  if (aborted(abort)) return;
  auto key_at = [&](uint32_t i) -> uint64_t {
    if (kFromA) return keys[i];
    return ((uint64_t)__float_as_uint(z_in[i]) << 32) | (uint64_t)prim[i];
  };
  const uint32_t n_long = *count;
  for (uint32_t li = 0; li < n_long; ++li) {
    const uint32_t t = list[li];
    const uint32_t beg = offsets[t], len = offsets[t + 1] - beg;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += gridDim.x * blockDim.x) {
      const uint32_t r = e / w, base = (r & ~1u) * w;
      const uint32_t lo = (r & 1u) ? base : base + w;          // partner run [lo, hi)
      const uint32_t hi = (r & 1u) ? base + w : min(base + 2 * w, len);
      const uint64_t key = key_at(beg + e);
      const float zo = kFromA ? z_out_tmp[beg + e] : z_out[beg + e];
      uint32_t below = 0;   // keys of the partner run below `key`
      if (lo < hi) {
        uint32_t a = lo, b = hi;
        while (a < b) {
          const uint32_t m = (a + b) >> 1;
          if (key_at(beg + m) < key) a = m + 1; else b = m;
        }
        below = a - lo;
      }
      const uint32_t dst = beg + base + (e - r * w) + below;
      if (kFromA) {
        z_in[dst] = __uint_as_float((uint32_t)(key >> 32));
        prim[dst] = (uint32_t)key;
        z_out[dst] = zo;
      } else {
        keys[dst] = key;
        z_out_tmp[dst] = zo;
      }
    }
  }
}

// Final copy of long lists left in buffer A into the output arrays.
__global__ void k_long_copy(const uint32_t *offsets, const uint32_t *list, const uint32_t *count,
                            const uint64_t *keys, const float *z_out_tmp, float *z_in, uint32_t *prim, float *z_out,
                            const uint32_t *abort) {
  if (aborted(abort)) return;
  const uint32_t n_long = *count;
  for (uint32_t li = 0; li < n_long; ++li) {
    const uint32_t t = list[li];
    const uint32_t beg = offsets[t], len = offsets[t + 1] - beg;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += gridDim.x * blockDim.x) {
      const uint64_t key = keys[beg + e];
      z_in[beg + e] = __uint_as_float((uint32_t)(key >> 32));
      prim[beg + e] = (uint32_t)key;
      z_out[beg + e] = z_out_tmp[beg + e];
    }
  }
}

// Lists of length 0 or 1 need no sort: copy straight through.
__global__ void k_tile_copy_short(const uint32_t *offsets, uint32_t n_tiles, const uint64_t *keys,
                                  const float *z_out_in, float *z_in, float *z_out, uint32_t *prim,
                                  const uint32_t *abort) {
  if (aborted(abort)) return;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x) {
    uint32_t beg = offsets[t];
    if (offsets[t + 1] - beg == 1) {
      uint64_t key = keys[beg];
      z_in[beg] = __uint_as_float((uint32_t)(key >> 32));
      prim[beg] = (uint32_t)key;
      z_out[beg] = z_out_in[beg];
    }
  }
}

// ---- exclusive scan of uint32 (three passes) ----------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr uint32_t kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *s_warp, uint32_t &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  total = s_warp[(blockDim.x >> 5) - 1];
  uint32_t prev = warp > 0 ? s_warp[warp - 1] : 0u;
  uint32_t r = prev + x - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_blocks(const uint32_t *in, uint32_t *out, uint32_t n, uint32_t *block_sums, uint32_t *max_out) {
  __shared__ uint32_t s_warp[32];
  const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  uint32_t v[kScanItems], sum = 0, mx = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < n ? in[base + i] : 0u;
    sum += v[i];
    mx = max(mx, v[i]);
  }
  uint32_t total;
  uint32_t ex = block_excl_scan(sum, s_warp, total);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = ex;
    ex += v[i];
  }
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
  if (max_out) {
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(max_out, mx);
  }
}

// Scans the block sums in place (single CTA, any count) and writes the total.
__global__ void __launch_bounds__(kScanThreads)
k_scan_sums(uint32_t *sums, uint32_t n_blocks, uint32_t *total_out) {
  __shared__ uint32_t s_warp[32];
  uint32_t carry = 0;
  for (uint32_t base = 0; base < n_blocks; base += kScanThreads) {
    uint32_t i = base + threadIdx.x;
    uint32_t v = i < n_blocks ? sums[i] : 0u;
    uint32_t total;
    uint32_t ex = block_excl_scan(v, s_warp, total);
    if (i < n_blocks) sums[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_scan_add(uint32_t *out, uint32_t n, const uint32_t *block_sums, const uint32_t *total,
                           uint32_t *tail) {
  const uint32_t base = blockIdx.x * kScanTile;
  const uint32_t add = block_sums[blockIdx.x];
  for (uint32_t i = threadIdx.x; i < kScanTile; i += blockDim.x) {
    uint32_t k = base + i;
    if (k < n) out[k] += add;
  }
  if (tail && blockIdx.x == 0 && threadIdx.x == 0) *tail = *total;
}

void scan_u32(const uint32_t *in, uint32_t *out, uint32_t n, uint32_t *block_sums,
              uint32_t *total, uint32_t *max_out, uint32_t *tail, cudaStream_t s) {
  if (n == 0) {
    cudaMemsetAsync(total, 0, sizeof(uint32_t), s);
    if (tail) cudaMemsetAsync(tail, 0, sizeof(uint32_t), s);
    return;
  }
  uint32_t nb = (n + kScanTile - 1) / kScanTile;
  count_launch(), k_scan_blocks<<<nb, kScanThreads, 0, s>>>(in, out, n, block_sums, max_out);
  count_launch(), k_scan_sums<<<1, kScanThreads, 0, s>>>(block_sums, nb, total);
  count_launch(), k_scan_add<<<nb, 256, 0, s>>>(out, n, block_sums, total, tail);
}

uint32_t scan_block_count(uint32_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

void launch_prim_bounds(const Job *jobs, int n_jobs, uint32_t n_prims, uint32_t *cand_count,
                        int4 *rects, cudaStream_t s) {
  if (!n_prims) return;
  count_launch(), k_prim_bounds<<<(n_prims + 255) / 256, 256, 0, s>>>(jobs, n_jobs, n_prims, cand_count, rects);
}

void launch_cull_pairs(const Job *jobs, int n_jobs, const uint32_t *cand_off, uint32_t n_prims,
                       const uint32_t *cand_total, const int4 *rects, uint32_t *tile_count, Pair *pairs,
                       uint32_t pair_cap, uint32_t *pair_counter, int n_sm, cudaStream_t s, bool stri) {
  if (!n_prims) return;
  count_launch(), k_cull_pairs<false><<<n_sm * 8, kCullWarps * 32, 0, s>>>(jobs, n_jobs, cand_off, n_prims,
                                                                           cand_total, rects, tile_count, pairs,
                                                                           pair_cap, pair_counter);
  if (stri)
    count_launch(), k_cull_pairs<true><<<n_sm * 8, kCullWarps * 32, 0, s>>>(jobs, n_jobs, cand_off, n_prims,
                                                                            cand_total, rects, tile_count, pairs,
                                                                            pair_cap, pair_counter);
}

void launch_copy_short(const uint32_t *offsets, uint32_t n_segs, const uint64_t *keys, const float *z_out_tmp,
                       float *z_in, float *z_out, uint32_t *prim, cudaStream_t s, const uint32_t *abort) {
  if (!n_segs) return;
  count_launch(), k_tile_copy_short<<<(n_segs + 255) / 256, 256, 0, s>>>(offsets, n_segs, keys, z_out_tmp, z_in,
                                                                         z_out, prim, abort);
}

void launch_tile_sort_range(const uint32_t *offsets, uint32_t n_segs, uint32_t max_len, uint32_t min_len,
                            const uint64_t *keys, const float *z_out_tmp, float *z_in, float *z_out,
                            uint32_t *prim, int n_sm, cudaStream_t s, const uint32_t *abort) {
  // Short lists: up to kSortSmall entries (48 KB of shared memory), a CTA
  // per list; longer ones up to kSortLarge, fewer and larger CTAs.
  const uint32_t small = kSortSmall;
  if (max_len > min_len && min_len < small) {
    uint32_t cap = max_len < small ? max_len : small;
    uint32_t n2 = 1;
    while (n2 < cap) n2 <<= 1;
    size_t sm = (size_t)n2 * 12;
    count_launch(), k_tile_sort<<<n_segs < 65535u ? n_segs : 65535u, 256, sm, s>>>(offsets, n_segs, keys, z_out_tmp,
                                                                               z_in, z_out, prim, min_len, small,
                                                                               abort);
  }
  if (max_len > small) {
    const uint32_t cap = max_len < kSortLarge ? max_len : kSortLarge;   // longer lists: launch_long_sort
    uint32_t n2 = 1;
    while (n2 < cap) n2 <<= 1;
    size_t sm = (size_t)n2 * 12;
    count_launch(), k_tile_sort<<<n_sm, 1024, sm, s>>>(offsets, n_segs, keys, z_out_tmp, z_in, z_out, prim,
                                                       min_len > small ? min_len : small, kSortLarge, abort);
  }
}

void launch_long_sort(const uint32_t *offsets, uint32_t n_tiles, uint32_t max_len, uint64_t *keys,
                      float *z_out_tmp, float *z_in, float *z_out, uint32_t *prim, uint32_t *list,
                      uint32_t *count, int n_sm, cudaStream_t s, const uint32_t *abort) {
  if (max_len <= kSortLarge || !n_tiles) return;
  cudaMemsetAsync(count, 0, sizeof(uint32_t), s);
  count_launch(), k_long_lists<<<(n_tiles + 255) / 256, 256, 0, s>>>(offsets, n_tiles, list, count, abort);
  count_launch(), k_chunk_sort<<<n_sm, 1024, (size_t)kSortLarge * 12, s>>>(offsets, list, count, keys, z_out_tmp,
                                                                           abort);
  bool in_a = true;
  for (uint32_t w = kSortLarge; w < max_len; w <<= 1) {
    if (in_a)
      count_launch(), k_merge_pass<true><<<n_sm * 4, 256, 0, s>>>(offsets, list, count, w, keys, z_out_tmp, z_in,
                                                                  prim, z_out, abort);
    else
      count_launch(), k_merge_pass<false><<<n_sm * 4, 256, 0, s>>>(offsets, list, count, w, keys, z_out_tmp, z_in,
                                                                   prim, z_out, abort);
    in_a = !in_a;
  }
  if (in_a)
    count_launch(), k_long_copy<<<n_sm * 4, 256, 0, s>>>(offsets, list, count, keys, z_out_tmp, z_in, prim, z_out,
                                                         abort);
}

void launch_scatter_sort(const Pair *pairs, const uint32_t *pair_counter, uint32_t pair_cap,
                         const uint32_t *offsets, uint32_t n_tiles, uint32_t max_overlap,
                         uint64_t *keys, float *z_out_tmp, float *z_in, float *z_out, uint32_t *prim,
                         int n_sm, cudaStream_t s, const uint32_t *abort, uint32_t *long_list,
                         uint32_t *long_count) {
  count_launch(), k_scatter<<<n_sm * 8, 256, 0, s>>>(pairs, pair_counter, pair_cap, offsets, keys, z_out_tmp, abort);
  if (!n_tiles) return;
  launch_copy_short(offsets, n_tiles, keys, z_out_tmp, z_in, z_out, prim, s, abort);
  if (max_overlap > 1)
    launch_tile_sort_range(offsets, n_tiles, max_overlap, 1, keys, z_out_tmp, z_in, z_out, prim, n_sm, s, abort);
  if (max_overlap > kSortLarge && long_list && long_count)
    launch_long_sort(offsets, n_tiles, max_overlap, keys, z_out_tmp, z_in, z_out, prim, long_list, long_count,
                     n_sm, s, abort);
}

void launch_check_capacity(const uint32_t *pair_counter, uint32_t pair_cap, const uint32_t *max_overlap,
                           uint32_t overlap_cap, uint32_t *status, cudaStream_t s) {
  count_launch(), k_check_capacity<<<1, 32, 0, s>>>(pair_counter, pair_cap, max_overlap, overlap_cap, status);
}

cudaError_t cull_set_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_tile_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)((size_t)kSortLarge * 12));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_chunk_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)((size_t)kSortLarge * 12));
}

}  // namespace st
