// st_prep.cpp -- host preparation of a blobtree structure (runs once per tree
// structure; primitive parameter edits never re-run it).
//
//   post-order linearisation .............. Sec. 4 (nodes stored after their children)
//   isLeft / ignoreMod .................... Sec. 4 bitfield, Sec. 9
//   fast ancestor pointers ................ Sec. 7.2, cuts of Sec. 9
//   ranges of interest .................... Sec. 5 (root (-inf, 0], R_o U R_p)
//   evaluation stack depth ................ Sec. 10, register and stack budget
#include <cmath>
#include <cstring>
#include <sstream>

#include "st_internal.h"

namespace st {

bool is_prim_kind(int k) {
  return k == ST_PRIM_SPHERE || k == ST_PRIM_RBOX || k == ST_PRIM_CAPSULE || k == ST_PRIM_TORUS ||
         k == ST_PRIM_SCONE || k == ST_PRIM_ELLIPSOID || k == ST_PRIM_RTRI || k == ST_PRIM_QUADRIC;
}

// Triangle frame in FP64 from a description record: edges e0 = b - a,
// e1 = c - b, e2 = a - c, unit normal n = e0 x (c - a) / |.|, and the
// in-plane outward edge normals m_i = e_i x n.  Returns |e0 x (c - a)|.
static double tri_frame(const float *q, double e[3][3], double n[3], double m[3][3]) {
  for (int k = 0; k < 3; ++k) {
    e[0][k] = (double)q[3 + k] - q[k];
    e[1][k] = (double)q[6 + k] - q[3 + k];
    e[2][k] = (double)q[k] - q[6 + k];
  }
  const double ca[3] = {-e[2][0], -e[2][1], -e[2][2]};
  double c[3] = {e[0][1] * ca[2] - e[0][2] * ca[1], e[0][2] * ca[0] - e[0][0] * ca[2],
                 e[0][0] * ca[1] - e[0][1] * ca[0]};
  const double len = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
  for (int k = 0; k < 3; ++k) n[k] = len > 0.0 ? c[k] / len : 0.0;
  for (int i = 0; i < 3; ++i) {
    m[i][0] = e[i][1] * n[2] - e[i][2] * n[1];
    m[i][1] = e[i][2] * n[0] - e[i][0] * n[2];
    m[i][2] = e[i][0] * n[1] - e[i][1] * n[0];
  }
  return len;
}

// Bounded quadric in FP64: rotation rows M (world -> local, the transpose of
// the unit quaternion's rotation) and the gradient bound G of q over the box.
static double quadric_frame(const float *q, double M[3][3]) {
  double w = q[3], x = q[4], y = q[5], z = q[6];
  const double nq = std::sqrt(w * w + x * x + y * y + z * z);
  if (nq > 0.0) { w /= nq; x /= nq; y /= nq; z /= nq; }
  const double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)},
                          {2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)},
                          {2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[i][j] = R[j][i];
  const double g0 = 2.0 * std::fabs((double)q[10]) * q[7], g1 = 2.0 * std::fabs((double)q[11]) * q[8];
  const double g2 = 2.0 * std::fabs((double)q[12]) * q[9] + std::fabs((double)q[13]);
  return std::sqrt(g0 * g0 + g1 * g1 + g2 * g2);
}

const char *prim_record_error(int kind, const float *q) {
  auto norm3 = [](const float *a) {
    return std::sqrt((double)a[0] * a[0] + (double)a[1] * a[1] + (double)a[2] * a[2]);
  };
  switch (kind) {
    case ST_PRIM_TORUS:
      if (!(norm3(q + 3) > 0.0)) return "torus: zero axis";
      if (!(q[6] >= 0.f) || !(q[7] > 0.f)) return "torus: needs R >= 0 and r > 0";
      return nullptr;
    case ST_PRIM_SCONE: {
      const float ba[3] = {q[3] - q[0], q[4] - q[1], q[5] - q[2]};
      if (!(q[6] >= 0.f) || !(q[7] >= 0.f) || !(q[6] + q[7] > 0.f)) return "sphere-cone: bad radii";
      if (!(norm3(ba) > std::fabs((double)q[6] - q[7]))) return "sphere-cone: one ball inside the other";
      return nullptr;
    }
    case ST_PRIM_ELLIPSOID:
      if (!(q[12] > 0.f) || !(q[13] > 0.f) || !(q[14] > 0.f)) return "ellipsoid: radii must be > 0";
      return nullptr;
    case ST_PRIM_RTRI: {
      double e[3][3], n[3], m[3][3];
      if (!(q[9] > 0.f)) return "rounded triangle: rounding must be > 0";
      if (!(tri_frame(q, e, n, m) > 0.0)) return "rounded triangle: collinear vertices";
      return nullptr;
    }
    case ST_PRIM_QUADRIC: {
      double M[3][3];
      if (!(norm3(q + 3) > 0.0 || q[6] != 0.f)) return "bounded quadric: zero quaternion";
      if (!(q[7] > 0.f) || !(q[8] > 0.f) || !(q[9] > 0.f)) return "bounded quadric: box half extents must be > 0";
      if (!(quadric_frame(q, M) > 0.0)) return "bounded quadric: alpha, beta, gamma and delta all zero";
      return nullptr;
    }
    default:
      return nullptr;
  }
}
static bool is_op_kind(int k) { return k >= ST_OP_UNION && k <= ST_OP_SHARP_DIFF; }
static bool is_compact(int k) { return k == ST_OP_UNION || k == ST_OP_INTER || k == ST_OP_DIFF; }

// ignoreMod of Sec. 9: bit 0 = ignore if the right operand is absent, bit 1 =
// ignore if the left operand is absent.
static uint32_t ignore_mode(int k) {
  switch (k) {
    case ST_OP_INTER: case ST_OP_SHARP_INTER: return 3;
    case ST_OP_DIFF: case ST_OP_SHARP_DIFF: return 2;
    default: return 0;
  }
}

void prim_words(int kind, const float *q, float *w) {
  std::memset(w, 0, sizeof(float) * 4 * rec_words(kind));
  if (kind == ST_PRIM_SPHERE) {
    w[0] = q[0]; w[1] = q[1]; w[2] = q[2]; w[3] = q[3];
  } else if (kind == ST_PRIM_RBOX) {
    w[0] = q[0]; w[1] = q[1]; w[2] = q[2]; w[3] = q[15];
    for (int i = 0; i < 3; ++i) {
      w[4 + 4 * i + 0] = q[3 + 3 * i];
      w[4 + 4 * i + 1] = q[4 + 3 * i];
      w[4 + 4 * i + 2] = q[5 + 3 * i];
      w[4 + 4 * i + 3] = q[12 + i];
    }
  } else if (kind == ST_PRIM_CAPSULE) {
    w[0] = q[0]; w[1] = q[1]; w[2] = q[2]; w[3] = q[6];
    w[4] = q[3]; w[5] = q[4]; w[6] = q[5]; w[7] = 0.f;
    float bx = q[3] - q[0], by = q[4] - q[1], bz = q[5] - q[2];
    float bb = (bx * bx + by * by) + bz * bz;
    w[8] = bx; w[9] = by; w[10] = bz; w[11] = bb > 0.f ? 1.0f / bb : 0.f;
  } else if (kind == ST_PRIM_TORUS) {
    // unit axis in FP64, rounded once
    const double n = std::sqrt((double)q[3] * q[3] + (double)q[4] * q[4] + (double)q[5] * q[5]);
    w[0] = q[0]; w[1] = q[1]; w[2] = q[2]; w[3] = q[7];
    for (int k = 0; k < 3; ++k) w[4 + k] = (float)(q[3 + k] / n);
    w[7] = q[6];
  } else if (kind == ST_PRIM_SCONE) {
    const double ba[3] = {(double)q[3] - q[0], (double)q[4] - q[1], (double)q[5] - q[2]};
    const double h = std::sqrt(ba[0] * ba[0] + ba[1] * ba[1] + ba[2] * ba[2]);
    const double sn = ((double)q[6] - q[7]) / h, cs = std::sqrt(1.0 - sn * sn);
    w[0] = q[0]; w[1] = q[1]; w[2] = q[2]; w[3] = q[6];
    w[4] = q[3]; w[5] = q[4]; w[6] = q[5]; w[7] = q[7];
    for (int k = 0; k < 3; ++k) w[8 + k] = (float)(ba[k] / h);
    w[11] = (float)h;
    w[12] = (float)sn; w[13] = (float)cs; w[14] = (float)(cs * h); w[15] = 0.f;
  } else if (kind == ST_PRIM_RTRI) {
    double e[3][3], n[3], m[3][3];
    tri_frame(q, e, n, m);
    w[0] = q[0]; w[1] = q[1]; w[2] = q[2]; w[3] = q[9];
    for (int i = 0; i < 3; ++i) {
      const double ee = e[i][0] * e[i][0] + e[i][1] * e[i][1] + e[i][2] * e[i][2];
      for (int k = 0; k < 3; ++k) w[4 + 4 * i + k] = (float)e[i][k];
      w[4 + 4 * i + 3] = (float)(1.0 / ee);
    }
    for (int k = 0; k < 3; ++k) {
      w[16 + k] = (float)n[k];
      w[20 + k] = (float)m[0][k];
      w[24 + k] = (float)m[1][k];
    }
    w[19] = (float)m[2][0]; w[23] = (float)m[2][1]; w[27] = (float)m[2][2];
  } else if (kind == ST_PRIM_QUADRIC) {
    double M[3][3];
    const double G = quadric_frame(q, M);
    w[0] = q[0]; w[1] = q[1]; w[2] = q[2]; w[3] = (float)((double)q[14] / G);
    for (int i = 0; i < 3; ++i) {
      for (int k = 0; k < 3; ++k) w[4 + 4 * i + k] = (float)M[i][k];
      w[4 + 4 * i + 3] = q[7 + i];
    }
    for (int k = 0; k < 4; ++k) w[16 + k] = (float)((double)q[10 + k] / G);
  } else {   // ellipsoid
    const float rmin = std::fmin(q[12], std::fmin(q[13], q[14]));
    w[0] = q[0]; w[1] = q[1]; w[2] = q[2]; w[3] = rmin;
    for (int i = 0; i < 3; ++i) {
      w[4 + 4 * i + 0] = q[3 + 3 * i];
      w[4 + 4 * i + 1] = q[4 + 3 * i];
      w[4 + 4 * i + 2] = q[5 + 3 * i];
      w[4 + 4 * i + 3] = q[12 + i];
      w[16 + i] = (float)(1.0 / (double)q[12 + i]);
    }
    w[19] = 0.f;
  }
}

static void prim_bounds(int kind, const float *q, double lo[3], double hi[3]) {
  if (kind == ST_PRIM_SPHERE) {
    for (int j = 0; j < 3; ++j) { lo[j] = (double)q[j] - q[3]; hi[j] = (double)q[j] + q[3]; }
  } else if (kind == ST_PRIM_RBOX) {
    for (int j = 0; j < 3; ++j) {
      double e = 0;
      for (int i = 0; i < 3; ++i) e += std::fabs((double)q[3 + 3 * i + j]) * ((double)q[12 + i] + q[15]);
      lo[j] = q[j] - e; hi[j] = q[j] + e;
    }
  } else if (kind == ST_PRIM_CAPSULE) {
    for (int j = 0; j < 3; ++j) {
      double a = q[j], b = q[3 + j];
      lo[j] = std::fmin(a, b) - q[6]; hi[j] = std::fmax(a, b) + q[6];
    }
  } else if (kind == ST_PRIM_TORUS) {
    const double n = std::sqrt((double)q[3] * q[3] + (double)q[4] * q[4] + (double)q[5] * q[5]);
    for (int j = 0; j < 3; ++j) {
      const double a = q[3 + j] / n;
      const double e = (double)q[6] * std::sqrt(std::fmax(0.0, 1.0 - a * a)) + q[7];
      lo[j] = q[j] - e; hi[j] = q[j] + e;
    }
  } else if (kind == ST_PRIM_SCONE) {
    for (int j = 0; j < 3; ++j) {
      lo[j] = std::fmin((double)q[j] - q[6], (double)q[3 + j] - q[7]);
      hi[j] = std::fmax((double)q[j] + q[6], (double)q[3 + j] + q[7]);
    }
  } else if (kind == ST_PRIM_RTRI) {
    for (int j = 0; j < 3; ++j) {
      lo[j] = std::fmin((double)q[j], std::fmin((double)q[3 + j], (double)q[6 + j])) - q[9];
      hi[j] = std::fmax((double)q[j], std::fmax((double)q[3 + j], (double)q[6 + j])) + q[9];
    }
  } else if (kind == ST_PRIM_QUADRIC) {   // inside its clipping box
    double M[3][3];
    quadric_frame(q, M);
    for (int j = 0; j < 3; ++j) {
      double e = 0;
      for (int i = 0; i < 3; ++i) e += std::fabs(M[i][j]) * q[7 + i];
      lo[j] = q[j] - e; hi[j] = q[j] + e;
    }
  } else {   // ellipsoid: inside its oriented box of half extents r
    for (int j = 0; j < 3; ++j) {
      double e = 0;
      for (int i = 0; i < 3; ++i) e += std::fabs((double)q[3 + 3 * i + j]) * q[12 + i];
      lo[j] = q[j] - e; hi[j] = q[j] + e;
    }
  }
}

int prepare(const st_scene_desc &d, Prep &p, std::string &err) {
  const int n = d.n_nodes;
  auto fail = [&](const std::string &m) { err = m; return ST_ERR_INVALID; };
  if (n < 1 || n > ST_MAX_NODES) return fail("n_nodes out of range");
  if (!d.kind || !d.left || !d.right || !d.params) return fail("null description array");
  if (d.root < 0 || d.root >= n) return fail("root index out of range");
  std::vector<int32_t> par(n, -1), isl(n, 0);
  int n_prims = 0;
  for (int i = 0; i < n; ++i) {
    int k = d.kind[i];
    if (is_prim_kind(k)) {
      if (d.left[i] != -1 || d.right[i] != -1) return fail("primitive with children");
      if (const char *e = prim_record_error(k, d.params + (size_t)i * ST_REC_FLOATS)) {
        std::ostringstream s; s << "node " << i << ": " << e;
        return fail(s.str());
      }
      ++n_prims;
      if (k == ST_PRIM_RTRI) p.has_stri = true;
      if (k != ST_PRIM_SPHERE && k != ST_PRIM_RBOX && k != ST_PRIM_CAPSULE) p.has_further = true;
      if (k == ST_PRIM_RTRI || k == ST_PRIM_QUADRIC) p.has_rtri_quadric = true;
      continue;
    }
    if (!is_op_kind(k)) {
      std::ostringstream s; s << "node " << i << ": kind " << k << " out of range";
      return fail(s.str());
    }
    int a = d.left[i], b = d.right[i];
    if (a < 0 || a >= n || b < 0 || b >= n || a == b) return fail("operator with bad children");
    if (par[a] != -1 || par[b] != -1) return fail("node with two parents");
    par[a] = i; isl[a] = 1;
    par[b] = i; isl[b] = 0;
    if (is_compact(k)) {
      float kk = d.params[(size_t)i * ST_REC_FLOATS + 0];
      float dd = d.params[(size_t)i * ST_REC_FLOATS + 1];
      if (!(kk > 0.f) || !(6.0f * dd - kk > 0.f)) return fail("compact operator needs k > 0 and 6 d_o > k");
    }
  }
  if (par[d.root] != -1) return fail("root has a parent");
  if (2 * n_prims - 1 != n) return fail("not a binary tree: n_nodes != 2 N - 1");

  // Iterative post-order from the root; reaching every node exactly once
  // (with the parent checks above) rules out cycles and forests.
  p.po_of_desc.assign(n, -1);
  p.desc_of_po.assign(n, -1);
  {
    std::vector<std::pair<int, int>> stk;
    stk.reserve(64);
    stk.push_back({d.root, 0});
    int counter = 0;
    while (!stk.empty()) {
      auto &top = stk.back();
      int v = top.first;
      if (is_prim_kind(d.kind[v]) || top.second == 2) {
        if (p.po_of_desc[v] != -1 || counter >= n) return fail("cycle in tree");
        p.po_of_desc[v] = counter;
        p.desc_of_po[counter] = v;
        ++counter;
        stk.pop_back();
        continue;
      }
      int child = top.second == 0 ? d.left[v] : d.right[v];
      top.second++;
      if ((int)stk.size() > n) return fail("cycle in tree");
      stk.push_back({child, 0});
    }
    if (counter != n) return fail("unreachable nodes");
  }

  p.parent.assign(n, -1);
  std::vector<int32_t> kind_po(n), isl_po(n);
  for (int a = 0; a < n; ++a) {
    int i = p.desc_of_po[a];
    kind_po[a] = d.kind[i];
    isl_po[a] = isl[i];
    p.parent[a] = par[i] < 0 ? -1 : p.po_of_desc[par[i]];
  }
  const int root = n - 1;

  // Ranges of interest, top-down (parents have larger addresses).
  p.roi.assign(n, 0.f);
  for (int a = root; a >= 0; --a) {
    int k = kind_po[a];
    if (is_prim_kind(k)) continue;
    int i = p.desc_of_po[a];
    float dc = p.roi[a];
    if (is_compact(k)) {
      float dop = d.params[(size_t)i * ST_REC_FLOATS + 1];
      if (dop > dc) dc = dop;
    }
    p.roi[p.po_of_desc[d.left[i]]] = dc;
    p.roi[p.po_of_desc[d.right[i]]] = dc;
  }

  // Fast ancestors, top-down in O(n): node P with parent A jumps over A iff A
  // is not the root, P and A lie on the same side of their parents, and A
  // passes a lone operand from P's side through (no intersection, no
  // difference reached from its right operand); then fast(P) = fast(A).
  std::vector<uint32_t> fast(n, kNoAnc);
  for (int a = root - 1; a >= 0; --a) {
    int A = p.parent[a];
    uint32_t f = (uint32_t)A;
    if (A != root && isl_po[a] == isl_po[A]) {
      uint32_t m = ignore_mode(kind_po[A]);
      bool passes = !(m & (isl_po[a] ? 1u : 2u));
      if (passes) f = fast[A];
    }
    fast[a] = f;
  }

  // Nearest blocking ancestor, top-down: the first ancestor at which a lone
  // operand coming up from this node's side is not passed through (Sec. 9
  // usage rule); a usage bit climbing from node v to an ancestor w survives
  // iff blk(v) >= w.
  p.blk.assign(n, kNoAnc);
  for (int a = root - 1; a >= 0; --a) {
    const int A = p.parent[a];
    const uint32_t m = ignore_mode(kind_po[A]);
    const bool passes = !(m & (isl_po[a] ? 1u : 2u));
    p.blk[a] = passes ? p.blk[A] : (uint32_t)A;
  }
  // Binary-lifting ancestor table: lift[k][a] = ancestor 2^k levels above a.
  {
    std::vector<int32_t> lvl(n, 0);
    int max_lvl = 0;
    for (int a = root - 1; a >= 0; --a) {
      lvl[a] = lvl[p.parent[a]] + 1;
      max_lvl = std::max(max_lvl, lvl[a]);
    }
    int K = 1;
    while ((1 << K) <= max_lvl) ++K;
    p.lift_levels = K;
    p.lift.assign((size_t)K * n, 0xFFFFFFFFu);
    for (int a = 0; a < n; ++a) p.lift[a] = p.parent[a] < 0 ? 0xFFFFFFFFu : (uint32_t)p.parent[a];
    for (int k = 1; k < K; ++k)
      for (int a = 0; a < n; ++a) {
        const uint32_t mid = p.lift[(size_t)(k - 1) * n + a];
        p.lift[(size_t)k * n + a] = mid == 0xFFFFFFFFu ? mid : p.lift[(size_t)(k - 1) * n + mid];
      }
  }

  // Post-order evaluation stack depth (Algorithm 3).
  std::vector<int32_t> depth(n, 1);
  for (int a = 0; a < n; ++a) {
    if (is_prim_kind(kind_po[a])) continue;
    int i = p.desc_of_po[a];
    int l = p.po_of_desc[d.left[i]], r = p.po_of_desc[d.right[i]];
    depth[a] = std::max(depth[l], depth[r] + 1);
  }
  p.stack_depth = depth[root];

  p.blob.assign(n, 0);
  for (int a = 0; a < n; ++a) {
    int k = kind_po[a];
    bool pr = is_prim_kind(k);
    p.blob[a] = make_blob(pr ? 1u : 0u, (uint32_t)k, pr ? 0u : ignore_mode(k), (uint32_t)isl_po[a],
                          a == root ? kNoAnc : fast[a]);
  }

  // Records and per-primitive arrays.
  p.rec_off.assign(n, 0);
  p.rec.clear();
  p.prim_addr.clear();
  p.d_prim.clear();
  p.prim_desc.clear();
  p.prim_index.assign(n, 0xFFFFFFFFu);
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int a = 0; a < n; ++a) {
    int i = p.desc_of_po[a];
    int k = kind_po[a];
    const float *q = d.params + (size_t)i * ST_REC_FLOATS;
    p.rec_off[a] = (uint32_t)(p.rec.size() / 4);
    if (is_prim_kind(k)) {
      float w[4 * kMaxRecWords];
      prim_words(k, q, w);
      p.rec.insert(p.rec.end(), w, w + 4 * rec_words(k));
      p.prim_index[a] = (uint32_t)p.prim_addr.size();
      p.prim_addr.push_back((uint32_t)a);
      p.d_prim.push_back(p.roi[a]);
      p.prim_desc.push_back(i);
      double l[3], h[3];
      prim_bounds(k, q, l, h);
      for (int j = 0; j < 3; ++j) { lo[j] = std::fmin(lo[j], l[j]); hi[j] = std::fmax(hi[j], h[j]); }
    } else if (is_compact(k)) {
      float kk = q[0], dd = q[1];
      p.rec.push_back(kk);
      p.rec.push_back(dd);
      p.rec.push_back(6.0f / (6.0f * dd - kk));
      p.rec.push_back(1.0f / kk);
    } else {
      for (int j = 0; j < 4; ++j) p.rec.push_back(0.f);
    }
  }
  if (p.rec.size() / 4 > kViewOffMask) return fail("too many record words");
  double s = 0, e = 0;
  for (int j = 0; j < 3; ++j) {
    s += (hi[j] - lo[j]) * (hi[j] - lo[j]);
    e = std::fmax(e, hi[j] - lo[j]);
  }
  p.diameter = std::sqrt(s);
  p.extent = e;
  return ST_OK;
}

void camera_basis(const st_camera &c, DevCamera &out) {
  double e[3] = {c.eye[0], c.eye[1], c.eye[2]};
  double up[3] = {c.up[0], c.up[1], c.up[2]};
  double F[3] = {(double)c.target[0] - e[0], (double)c.target[1] - e[1], (double)c.target[2] - e[2]};
  double nf = std::sqrt((F[0] * F[0] + F[1] * F[1]) + F[2] * F[2]);
  for (int j = 0; j < 3; ++j) F[j] = F[j] / nf;
  double R[3] = {F[1] * up[2] - F[2] * up[1], F[2] * up[0] - F[0] * up[2], F[0] * up[1] - F[1] * up[0]};
  double nr = std::sqrt((R[0] * R[0] + R[1] * R[1]) + R[2] * R[2]);
  for (int j = 0; j < 3; ++j) R[j] = R[j] / nr;
  double U[3] = {R[1] * F[2] - R[2] * F[1], R[2] * F[0] - R[0] * F[2], R[0] * F[1] - R[1] * F[0]};
  double th = std::tan((double)c.vfov_deg * M_PI / 360.0);
  double aspect = (double)c.width / (double)c.height;
  for (int j = 0; j < 3; ++j) {
    out.o[j] = (float)e[j];
    out.F[j] = (float)F[j];
    out.R[j] = (float)(R[j] * th * aspect);
    out.U[j] = (float)(U[j] * th);
  }
  out.W = c.width;
  out.H = c.height;
}

}  // namespace st

extern "C" int st_prep_tree(const st_scene_desc *desc, int32_t *po_of_desc, uint32_t *blob,
                            int32_t *parent, float *roi) {
  if (!desc) { st::set_error("null description"); return ST_ERR_INVALID; }
  st::Prep p;
  std::string err;
  int rc = st::prepare(*desc, p, err);
  if (rc != ST_OK) { st::set_error(err); return rc; }
  const size_t n = (size_t)desc->n_nodes;
  if (po_of_desc) std::memcpy(po_of_desc, p.po_of_desc.data(), n * sizeof(int32_t));
  if (blob) std::memcpy(blob, p.blob.data(), n * sizeof(uint32_t));
  if (parent) std::memcpy(parent, p.parent.data(), n * sizeof(int32_t));
  if (roi) std::memcpy(roi, p.roi.data(), n * sizeof(float));
  return p.stack_depth;
}
