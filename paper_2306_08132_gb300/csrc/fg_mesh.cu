// Mesh objects (Sec. III-B): a watertight triangle mesh queried directly through
// a bounding volume hierarchy, with the Phong-smoothed SDF.  Everything here runs
// on the host at object creation: validation, normals, pseudonormals, the BVH,
// and the data of the certified local search (faces on the convex hull, face
// adjacency, vertex rings, a coarse table of start faces); the device arrays are
// then copied once (one allocation per object).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include "fg_internal.h"

namespace fg {

namespace {

constexpr int kLeafFaces = 4;
constexpr int kStartCells = 32;    // nodes of the start-face table along the longest axis
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

// Closest point of p on triangle (a, b, c) (double precision, Voronoi regions of
// the vertices, edges and face): squared distance.
double closest_sq(const Vec& p, const Vec& a, const Vec& b, const Vec& c) {
  const Vec ab = sub(b, a), ac = sub(c, a), ap = sub(p, a), bp = sub(p, b), cp = sub(p, c);
  const double d1 = dot(ab, ap), d2 = dot(ac, ap), d3 = dot(ab, bp), d4 = dot(ac, bp), d5 = dot(ab, cp),
               d6 = dot(ac, cp);
  const double vc = d1 * d4 - d3 * d2, vb = d5 * d2 - d1 * d6, va = d3 * d6 - d5 * d4;
  Vec q;
  if (d1 <= 0 && d2 <= 0) q = a;
  else if (d3 >= 0 && d4 <= d3) q = b;
  else if (vc <= 0 && d1 >= 0 && d3 <= 0) q = add(a, scale(ab, d1 / (d1 - d3)));
  else if (d6 >= 0 && d5 <= d6) q = c;
  else if (vb <= 0 && d2 >= 0 && d6 <= 0) q = add(a, scale(ac, d2 / (d2 - d6)));
  else if (va <= 0 && d4 - d3 >= 0 && d5 - d6 >= 0) q = add(b, scale(sub(c, b), (d4 - d3) / ((d4 - d3) + (d5 - d6))));
  else {
    const double den = 1.0 / (va + vb + vc);
    q = add(a, add(scale(ab, vb * den), scale(ac, vc * den)));
  }
  const Vec r = sub(p, q);
  return dot(r, r);
}

inline double box_sq(const Vec& p, const Node& n) {
  const double c[3] = {p.x, p.y, p.z};
  double s = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double d = std::max(std::max((double)n.lo[k] - c[k], c[k] - (double)n.hi[k]), 0.0);
    s += d * d;
  }
  return s;
}

// Closest face of p (position in BVH order), depth first over the host BVH.
int closest_face(const Builder& B, const Vec& p) {
  int stack[2 * kMaxDepth + 4];
  int sp = 0, node = 0, best = -1;
  double best_d2 = 1e300;
  for (;;) {
    const Node& n = B.nodes[node];
    if (n.count > 0) {
      for (int j = n.link; j < n.link + n.count; ++j) {
        const int f = B.order[j];
        const double d2 = closest_sq(p, B.V[B.F[3 * f]], B.V[B.F[3 * f + 1]], B.V[B.F[3 * f + 2]]);
        if (d2 < best_d2) {
          best_d2 = d2;
          best = j;
        }
      }
    } else {
      const int l = node + 1, r = n.link;
      const double dl = box_sq(p, B.nodes[l]), dr = box_sq(p, B.nodes[r]);
      const int nearc = dl <= dr ? l : r, farc = dl <= dr ? r : l;
      if (std::max(dl, dr) < best_d2) stack[sp++] = farc;
      if (std::min(dl, dr) < best_d2) {
        node = nearc;
        continue;
      }
    }
    bool found = false;
    while (sp > 0) {
      const int c = stack[--sp];
      if (box_sq(p, B.nodes[c]) < best_d2) {
        node = c;
        found = true;
        break;
      }
    }
    if (!found) break;
  }
  return best;
}

// True when no vertex of the mesh lies more than tol outside the plane n . x = off
// (the face is then on the boundary of the convex hull): a search over the BVH
// boxes, whose highest corner bounds n . x of everything inside them.
bool below_plane(const Builder& B, const Vec& n, double off, double tol) {
  int stack[2 * kMaxDepth + 4];
  int sp = 0;
  stack[sp++] = 0;
  while (sp > 0) {
    const Node& nd = B.nodes[stack[--sp]];
    const double ub = std::max(n.x * nd.lo[0], n.x * nd.hi[0]) + std::max(n.y * nd.lo[1], n.y * nd.hi[1]) +
                      std::max(n.z * nd.lo[2], n.z * nd.hi[2]);
    if (ub <= off + tol) continue;
    if (nd.count > 0) {
      for (int j = nd.link; j < nd.link + nd.count; ++j) {
        const int f = B.order[j];
        for (int k = 0; k < 3; ++k)
          if (dot(n, B.V[B.F[3 * f + k]]) > off + tol) return false;
      }
    } else {
      const int self = (int)(&nd - B.nodes.data());
      stack[sp++] = self + 1;
      stack[sp++] = nd.link;
    }
  }
  return true;
}

fg_status mesh_invalid(const std::string& msg) {
  set_error("fg_sdf_create_mesh: " + msg);
  return FG_ERR_INVALID;
}

}  // namespace

}  // namespace fg

using namespace fg;

namespace fg {

namespace {

// Everything the host builds for a mesh object: the device image (one float4 array)
// and where its parts start, the start-face grid, the Phong shift bound, and counts.
struct MeshBuild {
  std::vector<float4> buf;
  size_t tri = 0, nrm = 0, wing = 0, ring = 0, start = 0;   // offsets in float4
  double blo[3] = {0.0, 0.0, 0.0}, sh = 1.0, shift = 0.0;
  int sn[3] = {0, 0, 0};
  int hull_faces = 0, fan_vertices = 0, nodes = 0, depth = 0;
};

fg_status build_mesh(const char* who, const float* vertices, int nv, const int* faces, int nf, float phong_alpha,
                     MeshBuild& M) {
  auto invalid = [&](const std::string& msg) {
    set_error(std::string(who) + ": " + msg);
    return FG_ERR_INVALID;
  };
  if (!vertices || !faces) return invalid("NULL argument");
  if (nv < 4 || nf < 4) return invalid("a closed mesh needs at least 4 vertices and 4 faces");
  if (nf > (1 << 24) || nv > (1 << 24)) return invalid("more than 2^24 vertices or faces");
  if (!(phong_alpha >= 0.0f && phong_alpha <= 1.0f)) return invalid("phong_alpha must be in [0, 1]");
  std::vector<Vec> V(nv);
  for (int i = 0; i < nv; ++i) {
    const float* p = vertices + 3 * i;
    if (!std::isfinite(p[0]) || !std::isfinite(p[1]) || !std::isfinite(p[2])) return invalid("non-finite vertex");
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
    if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) return invalid("face index out of range");
    if (a == b || b == c || c == a) return invalid("face with a repeated vertex");
    const Vec n = cross(sub(V[b], V[a]), sub(V[c], V[a]));
    if (!(norm(n) > 1e-12 * extent * extent)) return invalid("degenerate (zero-area) face");
    fn[f] = unit(n);
    volume += dot(V[a], cross(V[b], V[c])) / 6.0;
    const int e[3][2] = {{a, b}, {b, c}, {c, a}};
    for (int k = 0; k < 3; ++k) {
      const uint64_t key = ((uint64_t)(uint32_t)e[k][0] << 32) | (uint32_t)e[k][1];
      if (!edge_owner.emplace(key, 3 * f + k).second)
        return invalid("a directed edge is used twice (inconsistent orientation or non-manifold)");
    }
  }
  if (!(volume > 0.0)) return invalid("faces must be counter-clockwise about the outward normal");
  std::vector<int> across(3 * (size_t)nf);
  for (int f = 0; f < nf; ++f) {
    for (int k = 0; k < 3; ++k) {
      const int u = F[3 * f + k], v = F[3 * f + (k + 1) % 3];
      auto it = edge_owner.find(((uint64_t)(uint32_t)v << 32) | (uint32_t)u);
      if (it == edge_owner.end()) return invalid("mesh is not watertight (an edge has one face)");
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
  std::vector<int> pos(nf);                       // BVH position of each face
  for (int j = 0; j < nf; ++j) pos[bld.order[j]] = j;

  // Certified local search.  A face is on the convex hull when no vertex lies more
  // than tol outside its plane (tol far below float32 rounding of a coordinate);
  // the mesh then lies inside the half-space of every hull face, so at a point of
  // the surface whose incident faces are all hull faces the convex hull's tangent
  // cone is the cone of the incident edges, and p - q in its normal cone proves q
  // the closest point of the whole mesh (up to tol).
  const double tol = 1e-9 * extent;
  std::vector<char> hull(nf);
  for (int f = 0; f < nf; ++f) hull[f] = below_plane(bld, fn[f], dot(fn[f], V[F[3 * f]]), tol);
  // vertex rings: per directed edge v -> u, the neighbour u and the face holding the edge
  std::vector<int> ring_start(nv + 1, 0);
  for (int i = 0; i < 3 * nf; ++i) ++ring_start[F[i] + 1];
  for (int v = 0; v < nv; ++v) ring_start[v + 1] += ring_start[v];
  std::vector<int> ring_u(3 * (size_t)nf), ring_f(3 * (size_t)nf), fill(ring_start.begin(), ring_start.end() - 1);
  std::vector<char> vert_hull(nv, 1);
  for (int f = 0; f < nf; ++f)
    for (int k = 0; k < 3; ++k) {
      const int v = F[3 * f + k];
      ring_u[fill[v]] = F[3 * f + (k + 1) % 3];
      ring_f[fill[v]++] = f;
      if (!hull[f]) vert_hull[v] = 0;
    }
  // Each ring in fan order: entry i's face (v, u_i, u_(i+1)) holds v -> u_i, so the two
  // faces on edge (v, u_i) are the faces of entries i and i - 1.  A vertex whose faces
  // form more than one fan keeps its ring unordered.
  std::vector<char> vert_fan(nv, 1);
  {
    std::vector<int> ou, of;
    std::vector<std::pair<int, int>> by_u;       // (neighbour, entry) of the current ring, sorted
    for (int v = 0; v < nv; ++v) {
      const int b = ring_start[v], m = ring_start[v + 1] - b;
      if (m == 0) continue;
      by_u.clear();
      for (int i = b; i < b + m; ++i) by_u.emplace_back(ring_u[i], i);
      std::sort(by_u.begin(), by_u.end());
      ou.assign(1, ring_u[b]);
      of.assign(1, ring_f[b]);
      for (int step = 1; step < m; ++step) {
        const int f = of.back(), u = ou.back();
        int w = -1;
        for (int t = 0; t < 3; ++t)
          if (F[3 * f + t] == u) w = F[3 * f + (t + 1) % 3];
        auto it = std::lower_bound(by_u.begin(), by_u.end(), std::make_pair(w, -1));
        const int next = it != by_u.end() && it->first == w ? it->second : -1;
        if (next < 0 || ring_f[next] == of[0]) break;
        ou.push_back(ring_u[next]);
        of.push_back(ring_f[next]);
      }
      if ((int)ou.size() == m) {
        std::copy(ou.begin(), ou.end(), ring_u.begin() + b);
        std::copy(of.begin(), of.end(), ring_f.begin() + b);
      } else {
        vert_fan[v] = 0;
      }
    }
  }
  // start faces: the closest face at the nodes of a coarse grid over the mesh's box
  // grown by its largest side on every side
  double blo[3] = {1e300, 1e300, 1e300}, bhi[3] = {-1e300, -1e300, -1e300};
  for (const Vec& p : V) {
    const double c[3] = {p.x, p.y, p.z};
    for (int a = 0; a < 3; ++a) {
      blo[a] = std::min(blo[a], c[a]);
      bhi[a] = std::max(bhi[a], c[a]);
    }
  }
  const double side = std::max(bhi[0] - blo[0], std::max(bhi[1] - blo[1], bhi[2] - blo[2]));
  const double sh = 3.0 * side / (kStartCells - 1);
  int sn[3];
  for (int a = 0; a < 3; ++a) {
    blo[a] -= side;
    sn[a] = std::min(kStartCells, (int)std::ceil((bhi[a] - blo[a] + side) / sh) + 1);
  }
  const size_t nstart = (size_t)sn[0] * sn[1] * sn[2];

  const size_t n_wing = 3 * (size_t)nf, n_ring = 3 * (size_t)nf, n_start = (nstart + 3) / 4;
  std::vector<float4> buf(2 * nn + 3 * (size_t)nf + 7 * (size_t)nf + n_wing + n_ring + n_start);
  float4* bvh = buf.data();
  float4* tri = bvh + 2 * nn;
  float4* nrm = tri + 3 * (size_t)nf;
  float4* wing = nrm + 7 * (size_t)nf;
  float4* ring = wing + n_wing;
  float4* start = ring + n_ring;
  for (size_t i = 0; i < nn; ++i) {
    const Node& n = bld.nodes[i];
    int link = n.link, count = n.count;
    float lw, hw;
    std::memcpy(&lw, &link, 4);
    std::memcpy(&hw, &count, 4);
    bvh[2 * i] = make_float4(n.lo[0], n.lo[1], n.lo[2], lw);
    bvh[2 * i + 1] = make_float4(n.hi[0], n.hi[1], n.hi[2], hw);
  }
  auto bits = [](int x) {
    float y;
    std::memcpy(&y, &x, 4);
    return y;
  };
  auto f4 = [](const Vec& v, float w) { return make_float4((float)v.x, (float)v.y, (float)v.z, w); };
  for (int j = 0; j < nf; ++j) {
    const int f = bld.order[j];
    for (int k = 0; k < 3; ++k) {
      const int v = F[3 * f + k], g = across[3 * f + k];
      // vertex k and the face across edge (k, k+1)
      tri[3 * j + k] = make_float4(vertices[3 * v], vertices[3 * v + 1], vertices[3 * v + 2], bits(pos[g]));
      // vertex normal and the ring of vertex k: first edge; edge pseudonormal and the
      // ring's length, bit 30 set when every face around the vertex is a hull face,
      // bit 29 when the ring is in fan order
      nrm[7 * j + k] = f4(vn[v], bits(ring_start[v]));
      const int len = ring_start[v + 1] - ring_start[v];
      nrm[7 * j + 4 + k] =
          f4(unit(add(fn[f], fn[g])), bits(len | (vert_hull[v] ? 1 << 30 : 0) | (vert_fan[v] ? 1 << 29 : 0)));
      // the vertex of g opposite edge (k, k+1); 1 when both faces are hull faces
      const int u = F[3 * f + (k + 1) % 3];
      int opp = F[3 * g];
      for (int t = 0; t < 3; ++t)
        if (F[3 * g + t] != v && F[3 * g + t] != u) opp = F[3 * g + t];
      wing[3 * j + k] = make_float4(vertices[3 * opp], vertices[3 * opp + 1], vertices[3 * opp + 2],
                                    bits(hull[f] && hull[g] ? 1 : 0));
    }
    nrm[7 * j + 3] = f4(fn[f], bits(hull[f] ? 1 : 0));   // face normal; 1 for a hull face
  }
  for (size_t i = 0; i < n_ring; ++i) {
    const int u = ring_u[i];
    ring[i] = make_float4(vertices[3 * u], vertices[3 * u + 1], vertices[3 * u + 2], bits(pos[ring_f[i]]));
  }
  {
    std::vector<int> sf(nstart);
    for (int z = 0; z < sn[2]; ++z)
      for (int y = 0; y < sn[1]; ++y)
        for (int x = 0; x < sn[0]; ++x)
          sf[((size_t)z * sn[1] + y) * sn[0] + x] = closest_face(bld, Vec{blo[0] + sh * x, blo[1] + sh * y, blo[2] + sh * z});
    std::memcpy(start, sf.data(), sizeof(int) * nstart);
  }
  for (int f = 0; f < nf; ++f) M.hull_faces += hull[f] ? 1 : 0;
  for (int v = 0; v < nv; ++v) M.fan_vertices += (vert_fan[v] && ring_start[v + 1] > ring_start[v]) ? 1 : 0;
  M.nodes = (int)nn;
  M.depth = bld.depth_reached;
  M.tri = tri - bvh;
  M.nrm = nrm - bvh;
  M.wing = wing - bvh;
  M.ring = ring - bvh;
  M.start = start - bvh;
  for (int a = 0; a < 3; ++a) {
    M.blo[a] = blo[a];
    M.sn[a] = sn[a];
  }
  M.sh = sh;
  M.shift = shift;
  M.buf = std::move(buf);
  return FG_OK;
}

}  // namespace

}  // namespace fg

extern "C" fg_status fg_sdf_create_mesh(const float* vertices, int nv, const int* faces, int nf, float phong_alpha,
                                        float mass, float inertia, fg_sdf** out) {
  if (!vertices || !faces || !out) return mesh_invalid("NULL argument");
  *out = nullptr;
  if (!(mass > 0.0f) || !(inertia > 0.0f) || !std::isfinite(mass) || !std::isfinite(inertia))
    return mesh_invalid("mass and inertia must be > 0");
  MeshBuild M;
  const fg_status st = build_mesh("fg_sdf_create_mesh", vertices, nv, faces, nf, phong_alpha, M);
  if (st != FG_OK) return st;
  fg_sdf* s = new (std::nothrow) fg_sdf;
  if (!s) return FG_ERR_OOM;
  std::memset(s, 0, sizeof(*s));
  s->bytes = sizeof(float4) * M.buf.size();
  float4* dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, s->bytes);
  if (e == cudaSuccess) e = cudaMemcpy(dev, M.buf.data(), s->bytes, cudaMemcpyHostToDevice);
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
  o.phong_shift = (float)(M.shift * (1.0 + 1e-5)) + 1e-7f;
  o.bvh = dev;
  o.tri = dev + M.tri;
  o.face_nrm = dev + M.nrm;
  o.wing = dev + M.wing;
  o.ring = dev + M.ring;
  o.start_face = reinterpret_cast<const int*>(dev + M.start);
  for (int a = 0; a < 3; ++a) {
    o.start_org[a] = (float)M.blo[a];
    o.start_n[a] = M.sn[a];
  }
  o.start_inv_h = (float)(1.0 / M.sh);
  o.inv_mass = 1.0f / mass;
  o.inv_inertia = 1.0f / inertia;
  o.h = 1.0f;          // unused by mesh queries
  o.inv_h = 1.0f;
  *out = s;
  return FG_OK;
}

extern "C" fg_status fg_mesh_describe(const float* vertices, int nv, const int* faces, int nf, int* out6) {
  if (!out6) {
    set_error("fg_mesh_describe: NULL argument");
    return FG_ERR_INVALID;
  }
  MeshBuild M;
  const fg_status st = build_mesh("fg_mesh_describe", vertices, nv, faces, nf, 0.0f, M);
  if (st != FG_OK) return st;
  out6[0] = nf;
  out6[1] = M.hull_faces;
  out6[2] = M.fan_vertices;
  out6[3] = M.nodes;
  out6[4] = M.depth;
  out6[5] = M.sn[0] * M.sn[1] * M.sn[2];
  return FG_OK;
}
