// Mesh objects (Sec. III-B): a watertight triangle mesh queried directly through
// a bounding volume hierarchy, with the Phong-smoothed SDF.  Everything here runs
// on the host at object creation: validation, normals, pseudonormals and the
// BVH; the device arrays are then copied once (one allocation per object).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "fg_internal.h"

namespace fg {

namespace {

constexpr int kLeafFaces = 4;
constexpr int kMaxDepth = 48;      // the device traversal keeps at most one entry per level

struct Vec {
  double x, y, z;
};
inline Vec sub(const Vec& a, const Vec& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline Vec add(const Vec& a, const Vec& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline Vec scale(const Vec& a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline double dot(const Vec& a, const Vec& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline Vec cross(const Vec& a, const Vec& b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double norm(const Vec& a) { return std::sqrt(dot(a, a)); }
inline Vec unit(const Vec& a) { return scale(a, 1.0 / norm(a)); }

struct Node {
  float lo[3], hi[3];
  int link;    // inner: right child; leaf: first face
  int count;   // faces in a leaf, 0 for an inner node
};

struct Builder {
  const std::vector<Vec>& V;
  const std::vector<int>& F;
  std::vector<int> order;          // face permutation (leaf ranges are contiguous)
  std::vector<Vec> centroid;
  std::vector<Node> nodes;
  int depth_reached = 0;

  Builder(const std::vector<Vec>& v, const std::vector<int>& f) : V(v), F(f) {
    const int nf = (int)F.size() / 3;
    order.resize(nf);
    centroid.resize(nf);
    for (int i = 0; i < nf; ++i) {
      order[i] = i;
      centroid[i] = scale(add(add(V[F[3 * i]], V[F[3 * i + 1]]), V[F[3 * i + 2]]), 1.0 / 3.0);
    }
  }

  int build(int begin, int end, int depth) {
    depth_reached = std::max(depth_reached, depth);
    const int idx = (int)nodes.size();
    nodes.push_back(Node{});
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = begin; i < end; ++i) {
      const int f = order[i];
      for (int k = 0; k < 3; ++k) {
        const Vec& p = V[F[3 * f + k]];
        const double c[3] = {p.x, p.y, p.z};
        for (int a = 0; a < 3; ++a) {
          lo[a] = std::min(lo[a], c[a]);
          hi[a] = std::max(hi[a], c[a]);
        }
      }
    }
    for (int a = 0; a < 3; ++a) {
      // float boxes rounded outwards so that they contain the float vertices
      nodes[idx].lo[a] = std::nextafter((float)lo[a], -INFINITY);
      nodes[idx].hi[a] = std::nextafter((float)hi[a], INFINITY);
    }
    if (end - begin <= kLeafFaces || depth >= kMaxDepth) {
      nodes[idx].link = begin;
      nodes[idx].count = end - begin;
      return idx;
    }
    // Split by the surface-area heuristic: over each axis, faces sorted by
    // centroid, the split k minimising area(left box) k + area(right box) (n - k)
    // (the expected number of faces a query visits is proportional to it).
    const int n = end - begin;
    int best_axis = 0, best_k = n / 2;
    double best_cost = 1e300;
    std::vector<int> sorted(n);
    std::vector<double> right_area(n + 1);
    auto box_area = [](const double lo[3], const double hi[3]) {
      const double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
      return 2.0 * (dx * dy + dy * dz + dz * dx);
    };
    for (int axis = 0; axis < 3; ++axis) {
      auto key = [&](int f) { return axis == 0 ? centroid[f].x : (axis == 1 ? centroid[f].y : centroid[f].z); };
      std::copy(order.begin() + begin, order.begin() + end, sorted.begin());
      std::sort(sorted.begin(), sorted.end(), [&](int a, int b) { return key(a) < key(b) || (key(a) == key(b) && a < b); });
      double rlo[3] = {1e300, 1e300, 1e300}, rhi[3] = {-1e300, -1e300, -1e300};
      for (int i = n - 1; i >= 1; --i) {             // right_area[i]: box of sorted[i..n)
        for (int k = 0; k < 3; ++k) {
          const Vec& p = V[F[3 * sorted[i] + k]];
          const double c[3] = {p.x, p.y, p.z};
          for (int a = 0; a < 3; ++a) {
            rlo[a] = std::min(rlo[a], c[a]);
            rhi[a] = std::max(rhi[a], c[a]);
          }
        }
        right_area[i] = box_area(rlo, rhi);
      }
      double llo[3] = {1e300, 1e300, 1e300}, lhi[3] = {-1e300, -1e300, -1e300};
      for (int i = 0; i < n - 1; ++i) {              // left box of sorted[0..i]
        for (int k = 0; k < 3; ++k) {
          const Vec& p = V[F[3 * sorted[i] + k]];
          const double c[3] = {p.x, p.y, p.z};
          for (int a = 0; a < 3; ++a) {
            llo[a] = std::min(llo[a], c[a]);
            lhi[a] = std::max(lhi[a], c[a]);
          }
        }
        const double cost = box_area(llo, lhi) * (i + 1) + right_area[i + 1] * (n - i - 1);
        if (cost < best_cost) {
          best_cost = cost;
          best_axis = axis;
          best_k = i + 1;
        }
      }
    }
    auto best_key = [&](int f) {
      return best_axis == 0 ? centroid[f].x : (best_axis == 1 ? centroid[f].y : centroid[f].z);
    };
    std::sort(order.begin() + begin, order.begin() + end,
              [&](int a, int b) { return best_key(a) < best_key(b) || (best_key(a) == best_key(b) && a < b); });
    const int mid = begin + best_k;
    build(begin, mid, depth + 1);                 // left child is idx + 1
    const int right = build(mid, end, depth + 1);
    nodes[idx].link = right;
    nodes[idx].count = 0;
    return idx;
  }
};

fg_status mesh_invalid(const std::string& msg) {
  set_error("fg_sdf_create_mesh: " + msg);
  return FG_ERR_INVALID;
}

}  // namespace

}  // namespace fg

using namespace fg;

extern "C" fg_status fg_sdf_create_mesh(const float* vertices, int nv, const int* faces, int nf, float phong_alpha,
                                        float mass, float inertia, fg_sdf** out) {
  if (!vertices || !faces || !out) return mesh_invalid("NULL argument");
  *out = nullptr;
  if (nv < 4 || nf < 4) return mesh_invalid("a closed mesh needs at least 4 vertices and 4 faces");
  if (nf > (1 << 24) || nv > (1 << 24)) return mesh_invalid("more than 2^24 vertices or faces");
  if (!(phong_alpha >= 0.0f && phong_alpha <= 1.0f)) return mesh_invalid("phong_alpha must be in [0, 1]");
  if (!(mass > 0.0f) || !(inertia > 0.0f) || !std::isfinite(mass) || !std::isfinite(inertia))
    return mesh_invalid("mass and inertia must be > 0");
  std::vector<Vec> V(nv);
  for (int i = 0; i < nv; ++i) {
    const float* p = vertices + 3 * i;
    if (!std::isfinite(p[0]) || !std::isfinite(p[1]) || !std::isfinite(p[2])) return mesh_invalid("non-finite vertex");
    V[i] = {p[0], p[1], p[2]};
  }
  std::vector<int> F(faces, faces + 3 * (size_t)nf);
  double extent = 0.0;
  for (const Vec& p : V) extent = std::max(extent, std::max(std::fabs(p.x), std::max(std::fabs(p.y), std::fabs(p.z))));
  // faces: indices, area, orientation (every directed edge once, its reverse once)
  std::unordered_map<uint64_t, int> edge_owner;
  edge_owner.reserve(3 * (size_t)nf * 2);
  std::vector<Vec> fn(nf);
  double volume = 0.0;
  for (int f = 0; f < nf; ++f) {
    const int a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
    if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) return mesh_invalid("face index out of range");
    if (a == b || b == c || c == a) return mesh_invalid("face with a repeated vertex");
    const Vec n = cross(sub(V[b], V[a]), sub(V[c], V[a]));
    if (!(norm(n) > 1e-12 * extent * extent)) return mesh_invalid("degenerate (zero-area) face");
    fn[f] = unit(n);
    volume += dot(V[a], cross(V[b], V[c])) / 6.0;
    const int e[3][2] = {{a, b}, {b, c}, {c, a}};
    for (int k = 0; k < 3; ++k) {
      const uint64_t key = ((uint64_t)(uint32_t)e[k][0] << 32) | (uint32_t)e[k][1];
      if (!edge_owner.emplace(key, 3 * f + k).second)
        return mesh_invalid("a directed edge is used twice (inconsistent orientation or non-manifold)");
    }
  }
  if (!(volume > 0.0)) return mesh_invalid("faces must be counter-clockwise about the outward normal");
  std::vector<int> across(3 * (size_t)nf);
  for (int f = 0; f < nf; ++f) {
    for (int k = 0; k < 3; ++k) {
      const int u = F[3 * f + k], v = F[3 * f + (k + 1) % 3];
      auto it = edge_owner.find(((uint64_t)(uint32_t)v << 32) | (uint32_t)u);
      if (it == edge_owner.end()) return mesh_invalid("mesh is not watertight (an edge has one face)");
      across[3 * f + k] = it->second / 3;
    }
  }
  // angle-weighted vertex normals (Phong interpolation and vertex pseudonormals)
  std::vector<Vec> vn(nv, Vec{0.0, 0.0, 0.0});
  for (int f = 0; f < nf; ++f) {
    for (int k = 0; k < 3; ++k) {
      const Vec& p0 = V[F[3 * f + k]];
      const Vec e1 = sub(V[F[3 * f + (k + 1) % 3]], p0), e2 = sub(V[F[3 * f + (k + 2) % 3]], p0);
      const double c = std::max(-1.0, std::min(1.0, dot(e1, e2) / (norm(e1) * norm(e2))));
      vn[F[3 * f + k]] = add(vn[F[3 * f + k]], scale(fn[f], std::acos(c)));
    }
  }
  for (int i = 0; i < nv; ++i)
    if (norm(vn[i]) > 0.0) vn[i] = unit(vn[i]);     // vertices used by no face keep a zero normal
  // Bound on the Phong point's shift from the flat closest point r* on face f:
  // r*_rho - r* = -a sum_x b_x ((r* - v_x) . n_x) n_x, so |.| <= a max over vertices x, y
  // of the face of |(v_y - v_x) . n_x| (linear in r*, extreme at the vertices).
  double shift = 0.0;
  for (int f = 0; f < nf; ++f)
    for (int x = 0; x < 3; ++x)
      for (int y = 0; y < 3; ++y)
        shift = std::max(shift, std::fabs(dot(sub(V[F[3 * f + y]], V[F[3 * f + x]]), vn[F[3 * f + x]])));
  shift *= phong_alpha;
  // BVH over faces
  Builder bld(V, F);
  bld.build(0, nf, 0);
  const size_t nn = bld.nodes.size();
  std::vector<float4> buf(2 * nn + 3 * (size_t)nf + 7 * (size_t)nf);
  float4* bvh = buf.data();
  float4* tri = bvh + 2 * nn;
  float4* nrm = tri + 3 * (size_t)nf;
  for (size_t i = 0; i < nn; ++i) {
    const Node& n = bld.nodes[i];
    int link = n.link, count = n.count;
    float lw, hw;
    std::memcpy(&lw, &link, 4);
    std::memcpy(&hw, &count, 4);
    bvh[2 * i] = make_float4(n.lo[0], n.lo[1], n.lo[2], lw);
    bvh[2 * i + 1] = make_float4(n.hi[0], n.hi[1], n.hi[2], hw);
  }
  auto f4 = [](const Vec& v) { return make_float4((float)v.x, (float)v.y, (float)v.z, 0.0f); };
  for (int j = 0; j < nf; ++j) {
    const int f = bld.order[j];
    for (int k = 0; k < 3; ++k) {
      tri[3 * j + k] = make_float4(vertices[3 * F[3 * f + k]], vertices[3 * F[3 * f + k] + 1],
                                   vertices[3 * F[3 * f + k] + 2], 0.0f);
      nrm[7 * j + k] = f4(vn[F[3 * f + k]]);
      nrm[7 * j + 4 + k] = f4(unit(add(fn[f], fn[across[3 * f + k]])));   // edge (k, k+1)
    }
    nrm[7 * j + 3] = f4(fn[f]);
  }
  fg_sdf* s = new (std::nothrow) fg_sdf;
  if (!s) return FG_ERR_OOM;
  std::memset(s, 0, sizeof(*s));
  s->bytes = sizeof(float4) * buf.size();
  float4* dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, s->bytes);
  if (e == cudaSuccess) e = cudaMemcpy(dev, buf.data(), s->bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(dev);
    delete s;
    return cuda_status(e, "fg_sdf_create_mesh: device copy");
  }
  s->mesh = dev;
  ObjDev& o = s->host;
  o.kind = kObjMesh;
  o.n_faces = nf;
  o.phong_alpha = phong_alpha;
  o.phong_shift = (float)(shift * (1.0 + 1e-5)) + 1e-7f;
  o.bvh = dev;
  o.tri = dev + 2 * nn;
  o.face_nrm = dev + 2 * nn + 3 * (size_t)nf;
  o.inv_mass = 1.0f / mass;
  o.inv_inertia = 1.0f / inertia;
  o.h = 1.0f;          // unused by mesh queries
  o.inv_h = 1.0f;
  *out = s;
  return FG_OK;
}
