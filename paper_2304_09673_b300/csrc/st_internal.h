// st_internal.h -- device-side data layout shared by the library's sources.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "st.h"

namespace st {

// ---- packed node word (Sec. 4 "blob" bitfield, own field order) -----------
constexpr uint32_t kAncBits = 23;
constexpr uint32_t kAncMask = (1u << kAncBits) - 1u;  // 0x7FFFFF = no ancestor
constexpr uint32_t kNoAnc = kAncMask;
__host__ __device__ inline uint32_t blob_anc(uint32_t b) { return b & kAncMask; }
__host__ __device__ inline uint32_t blob_isleft(uint32_t b) { return (b >> 23) & 1u; }
__host__ __device__ inline uint32_t blob_igm(uint32_t b) { return (b >> 24) & 3u; }
__host__ __device__ inline uint32_t blob_kind(uint32_t b) { return (b >> 26) & 31u; }
__host__ __device__ inline uint32_t blob_isprim(uint32_t b) { return b >> 31; }
__host__ __device__ inline uint32_t make_blob(uint32_t isprim, uint32_t kind, uint32_t igm,
                                              uint32_t isleft, uint32_t anc) {
  return (isprim << 31) | (kind << 26) | (igm << 24) | (isleft << 23) | (anc & kAncMask);
}

// ---- pruned-view node codes --------------------------------------------------
// A view entry is uint32: bits 27..31 code, bit 26 set when the record is
// read from the scene's global record array (else from the view's shared
// parameter cache), bits 0..25 record word offset.
enum ViewCode : uint32_t {
  V_SPHERE = 0, V_RBOX = 1, V_CAPSULE = 2,            // primitives (< V_FIRST_OP)
  V_UNION = 3, V_INTER = 4, V_DIFF = 5,               // compact smooth G_op
  V_SUNION = 6, V_SINTER = 7, V_SDIFF = 8,            // sharp CSG
  V_INF = 9, V_RIGHT = 10, V_LEFT = 11,               // usage rewrites (Sec. 9)
  V_TORUS = 12, V_SCONE = 13, V_ELLIPSOID = 14,       // further primitives
  V_RTRI = 15, V_QUADRIC = 16,
  // CTA-split evaluation of a view (st_trace.cu): a segment stream stores
  // the running value into the next output slot and pops; the top program
  // pushes and loads a stored value (one float2 per lane).  Never in a view.
  V_STORE = 17, V_LOAD = 18,
};
constexpr uint32_t V_FIRST_OP = 3;
// Primitive view codes: 0..2 and 12..16 (equal to the primitive kinds but
// for the bounded quadric, kind 11 -> code 16).
__host__ __device__ inline bool is_prim_code(uint32_t code) { return code < V_FIRST_OP || code >= V_TORUS; }
__host__ __device__ inline uint32_t prim_view_code(uint32_t kind) {
  return kind == (uint32_t)ST_PRIM_QUADRIC ? (uint32_t)V_QUADRIC : kind;
}
constexpr uint32_t kViewCodeShift = 27;
constexpr uint32_t kViewGlobal = 1u << 26;
constexpr uint32_t kViewOffMask = (1u << 26) - 1u;

// Record words (float4) per node kind.
//   sphere : [c, r]
//   rbox   : [c, r_round] [M row0, b.x] [M row1, b.y] [M row2, b.z]
//   capsule: [a, r] [b, 0] [b - a, 1/|b - a|^2]
//   torus  : [c, r] [unit axis, R]
//   sphere-cone: [a, r_a] [b, r_b] [u = (b - a) / h, h = |b - a|]
//                [sin, cos, cos h, 0] (sin = (r_a - r_b) / h: the side's
//                outward normal in the axial plane is (cos, sin))
//   ellipsoid: [c, min r] [M row0, r0] [M row1, r1] [M row2, r2]
//              [1/r0, 1/r1, 1/r2, 0]
//   rounded triangle: [a, r] [e0 = b - a, 1/|e0|^2] [e1 = c - b, 1/|e1|^2]
//              [e2 = a - c, 1/|e2|^2] [unit normal n, m2.x] [m0, m2.y]
//              [m1, m2.z] with m_i = e_i x n (outward edge normals in the
//              plane)
//   bounded quadric: [c, kappa'] [M row0, e0] [M row1, e1] [M row2, e2]
//              [alpha', beta', gamma', delta'] (M world->local rotation,
//              coefficients divided by the gradient bound G)
//   compact operator: [k, d_o, 6 / (6 d_o - k), 1 / k]
//   sharp operator  : [0, 0, 0, 0]
constexpr int kMaxRecWords = 8;   // record words of any node kind, at most
__host__ __device__ inline int rec_words(int kind) {
  switch (kind) {
    case ST_PRIM_RBOX: return 4;
    case ST_PRIM_CAPSULE: return 3;
    case ST_PRIM_TORUS: return 2;
    case ST_PRIM_SCONE: return 4;
    case ST_PRIM_ELLIPSOID: return 5;
    case ST_PRIM_RTRI: return 7;
    case ST_PRIM_QUADRIC: return 5;
    default: return 1;
  }
}

// Algorithmic FP32 flop counts per node evaluation (FMA = 2), counted from
// the formulas: sphere |p-c|-r; rounded box; capsule; compact operator (two
// smooth-operator evaluations, b_r and the range tests); sharp operator.
constexpr uint32_t kFlopsSphere = 11;
constexpr uint32_t kFlopsRbox = 40;
constexpr uint32_t kFlopsCapsule = 25;
constexpr uint32_t kFlopsTorus = 20;
constexpr uint32_t kFlopsScone = 27;
constexpr uint32_t kFlopsEllipsoid = 28;
constexpr uint32_t kFlopsRtri = 80;
constexpr uint32_t kFlopsQuadric = 55;
constexpr uint32_t kFlopsCompactOp = 30;
constexpr uint32_t kFlopsSharpOp = 2;
constexpr uint32_t kFlopsStep = 6;

// Near plane: rays start at planar depth kZNear; a ray whose first sample
// there is inside the solid (f < -eps) is a hit clipped at the near plane
// (depth kZNear |d|, no refinement).
constexpr float kZNear = 0.01f;

// ---- device views of a scene, camera, A-buffer and outputs ---------------------
struct DevScene {
  const uint32_t *blob;      // [n_nodes] packed node words, post-order
  const uint32_t *rec_off;   // [n_nodes] first record word of each node
  const float4 *rec;         // record words
  const uint32_t *prim_addr; // [n_prims] post-order address of primitive j
  const float *d_prim;       // [n_prims] range-of-interest bound (Sec. 5)
  const uint32_t *blk;       // [n_nodes] nearest ancestor that does not pass a
                             // lone operand from this node's side (kNoAnc: none)
  const uint32_t *lift;      // [lift_levels][n_nodes] ancestor 2^k levels up
                             // (level 0 = parent; 0xFFFFFFFF above the root)
  const uint32_t *prim_index;// [n_nodes] primitive index j of a primitive node
                             // (0xFFFFFFFF for operators)
  int32_t n_nodes, n_prims, stack_depth, lift_levels;
  float diameter, voi_pad;
};

struct DevCamera {
  float o[3], F[3], R[3], U[3];  // R and U pre-scaled (see st.h)
  int32_t W, H;
};

struct DevTiles {
  int32_t tile, tiles_x, tiles_y;
  const uint32_t *offsets;  // [n_tiles + 1]
  const float *z_in, *z_out;
  const uint32_t *prim;
};

struct DevOut {
  float *depth, *normal;
  uint32_t *evals;
  uint8_t *flags;
};

struct TraceParams {
  float eps, lipschitz, depth_slab, newton_clamp;
  int32_t max_steps, max_new, newton_iters, step_mode;
  float omega;      // relaxation factor of ST_STEP_OVERRELAX / ST_STEP_CROSSING
  float min_step;   // ST_STEP_CROSSING: shortest step, distance units
};

// One culling or tracing job (a scene seen by a camera).
struct Job {
  DevScene sc;
  DevCamera cam;
  DevTiles tl;
  DevOut out;
  TraceParams tp;
  uint32_t tile_base;   // first global tile index of this job
  uint32_t prim_base;   // first global primitive index of this job
  uint32_t cand_base;   // unused slot (alignment)
  uint32_t pad;
};

// ---- host preparation ----------------------------------------------------------
struct Prep {
  std::vector<int32_t> po_of_desc, desc_of_po, parent;
  std::vector<uint32_t> blob, rec_off, prim_addr;
  std::vector<uint32_t> blk;    // nearest blocking ancestor (see DevScene::blk)
  std::vector<uint32_t> lift;   // binary-lifting ancestor table (see DevScene::lift)
  int lift_levels = 1;
  std::vector<uint32_t> prim_index;   // see DevScene::prim_index
  std::vector<float> roi, d_prim, rec;  // rec: 4 floats per word
  std::vector<int32_t> prim_desc;       // description index of primitive j
  int stack_depth = 0;
  double diameter = 0;   // diagonal of the primitives' bounding box
  double extent = 0;     // its largest edge
  bool has_stri = false; // a rounded triangle (sphere-triangle volume) is present
  bool has_further = false;  // a primitive beyond sphere, rounded box and capsule
  bool has_rtri_quadric = false;  // a rounded triangle or a bounded quadric
  // kernel instance tier of the scene (TraceLaunch::further)
  int further_level() const { return has_rtri_quadric ? 2 : has_further ? 1 : 0; }
};

// Returns ST_OK or ST_ERR_INVALID with `err` set.
int prepare(const st_scene_desc &d, Prep &p, std::string &err);
// Record words of one primitive description record (host-side conversion).
void prim_words(int kind, const float *q, float *words /* 4 * rec_words */);
// Checks a primitive record's parameters; returns an error text or nullptr.
const char *prim_record_error(int kind, const float *q);
bool is_prim_kind(int kind);

void camera_basis(const st_camera &c, DevCamera &out);

void set_error(const std::string &msg);
// Host-side count of kernel launches issued by the library (a CUDA graph
// replay adds the kernel nodes it launches).
int count_launch();
void count_launches(uint64_t n);
uint64_t launches_so_far();
// Host-side count of device allocations (cudaMalloc) made by the library.
void count_device_alloc();

}  // namespace st
