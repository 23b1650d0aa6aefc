// C ABI entry points: validation, handles, error reporting and dispatch.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fg_internal.h"

namespace fg {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

fg_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return FG_OK;
  set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
  return e == cudaErrorMemoryAllocation ? FG_ERR_OOM : FG_ERR_CUDA;
}

int device_sm_count() {
  static int cached[64];
  static bool init[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (!init[dev]) {
    int n = 1;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = n > 0 ? n : 1;
    init[dev] = true;
  }
  return cached[dev];
}

ParamsDev params_from(const fg_params* p) {
  ParamsDev d;
  d.alpha = p->alpha_leak;
  d.dt = p->dt;
  d.V = p->v_test;
  d.mu = p->mu;
  d.lr = p->lr;
  d.r0 = p->r0;
  d.w_range = p->w_range;
  d.w_limit = p->w_limit;
  d.w_pen = p->w_pen;
  d.schedule = p->schedule;
  d.sim_steps = p->sim_steps;
  d.gauss_seidel = p->gauss_seidel;
  return d;
}

static fg_status invalid(const std::string& msg) {
  set_error(msg);
  return FG_ERR_INVALID;
}

// Allocation-failure injection for tests: -1 disarmed, else the number of
// allocation points still to pass before one fails.
static std::atomic<long long> g_alloc_countdown{-1};

bool alloc_fault() {
  long long v = g_alloc_countdown.load();
  while (v >= 0) {
    if (g_alloc_countdown.compare_exchange_weak(v, v - 1)) return v == 0;
  }
  return false;
}

static fg_status check_params(const fg_params* p) {
  if (!p) return invalid("params is NULL");
  if (!(p->dt > 0.0f) || !std::isfinite(p->dt)) return invalid("params.dt must be > 0");
  if (!(p->v_test >= 0.0f) || !std::isfinite(p->v_test)) return invalid("params.v_test must be >= 0");
  if (!(p->mu >= 0.0f) || !std::isfinite(p->mu)) return invalid("params.mu must be >= 0");
  if (!(p->alpha_leak >= 0.0f && p->alpha_leak <= 1.0f)) return invalid("params.alpha_leak must be in [0, 1]");
  if (!(p->r0 >= 0.0f) || !std::isfinite(p->r0)) return invalid("params.r0 must be >= 0");
  if (!std::isfinite(p->lr) || !std::isfinite(p->w_range) || !std::isfinite(p->w_limit) || !std::isfinite(p->w_pen))
    return invalid("params has a non-finite weight");
  if (p->schedule != 0 && p->schedule != 1) return invalid("params.schedule must be 0 or 1");
  if (p->sim_steps < 0 || p->sim_steps > FG_MAX_SIM_STEPS)
    return invalid("params.sim_steps must be in [0, FG_MAX_SIM_STEPS]");
  if (p->gauss_seidel != 0 && p->gauss_seidel != 1) return invalid("params.gauss_seidel must be 0 or 1");
  if (p->gauss_seidel && p->sim_steps != 0)
    return invalid("params.gauss_seidel needs sim_steps = 0 (the one-step metric)");
  return FG_OK;
}

}  // namespace fg

using namespace fg;

extern "C" {

fg_status fg_version(int* major, int* minor) {
  if (major) *major = 1;
  if (minor) *minor = 0;
  return FG_OK;
}

const char* fg_status_string(fg_status s) {
  switch (s) {
    case FG_OK: return "FG_OK";
    case FG_ERR_INVALID: return "FG_ERR_INVALID";
    case FG_ERR_OOM: return "FG_ERR_OOM";
    case FG_ERR_BUDGET: return "FG_ERR_BUDGET";
    case FG_ERR_TIMEOUT: return "FG_ERR_TIMEOUT";
    case FG_ERR_CUDA: return "FG_ERR_CUDA";
    case FG_ERR_BUSY: return "FG_ERR_BUSY";
    case FG_ERR_NOT_FOUND: return "FG_ERR_NOT_FOUND";
  }
  return "FG_ERR_UNKNOWN";
}

fg_status fg_test_fail_allocation(int after) {
  if (after < -1) return invalid("fg_test_fail_allocation: after must be >= -1");
  g_alloc_countdown.store(after);
  return FG_OK;
}

fg_status fg_last_error(char* buf, size_t n) {
  if (!buf || n == 0) return FG_ERR_INVALID;
  size_t k = g_last_error.size() < n - 1 ? g_last_error.size() : n - 1;
  std::memcpy(buf, g_last_error.data(), k);
  buf[k] = '\0';
  return FG_OK;
}

fg_status fg_hand_create(const fg_hand_desc* d, fg_hand** out) {
  if (!d || !out) return invalid("fg_hand_create: NULL argument");
  *out = nullptr;
  const int L = d->n_links, P = d->n_points;
  if (L < 1 || L > FG_MAX_LINKS) return invalid("fg_hand_create: n_links must be in [1, 32]");
  if (P < 1 || P > FG_MAX_POINTS) return invalid("fg_hand_create: n_points must be in [1, 2^20]");
  if (!d->parent || !d->T_fix || !d->pts_local || !d->link_of_point || (L > 1 && (!d->axis || !d->q_low || !d->q_up)))
    return invalid("fg_hand_create: NULL array in descriptor");
  if (d->parent[0] != -1) return invalid("fg_hand_create: parent[0] must be -1");
  HandDev H;
  std::memset(&H, 0, sizeof(H));
  H.L = L;
  H.J = L - 1;
  H.D = 6 + L - 1;
  H.P = P;
  H.parent[0] = -1;
  H.depth[0] = 0;
  for (int l = 1; l < L; ++l) {
    int p = d->parent[l];
    if (p < 0 || p >= l) return invalid("fg_hand_create: links must be in topological order (0 <= parent[l] < l)");
    H.parent[l] = p;
    H.depth[l] = H.depth[p] + 1;
    if (H.depth[l] > H.max_depth) H.max_depth = H.depth[l];
  }
  // subtree sizes and depth-first preorder check: descendants of l are exactly [l+1, l+size)
  int size[FG_MAX_LINKS];
  for (int l = 0; l < L; ++l) size[l] = 1;
  for (int l = L - 1; l >= 1; --l) size[H.parent[l]] += size[l];
  for (int l = 0; l < L; ++l) {
    H.subtree_end[l] = l + size[l];
    for (int k = l + 1; k < l + size[l]; ++k) {
      int a = k;
      while (a > l) a = H.parent[a];
      if (a != l) return invalid("fg_hand_create: links must be in depth-first preorder (contiguous subtrees)");
    }
  }
  for (int l = 0; l < L; ++l)
    for (int k = 0; k < 12; ++k) {
      float v = d->T_fix[12 * l + k];
      if (!std::isfinite(v)) return invalid("fg_hand_create: non-finite T_fix");
      H.T_fix[l][k] = v;
    }
  for (int l = 1; l < L; ++l) {
    float n2 = 0.0f;
    for (int k = 0; k < 3; ++k) {
      H.axis[l][k] = d->axis[3 * l + k];
      n2 += H.axis[l][k] * H.axis[l][k];
    }
    if (!(std::fabs(n2 - 1.0f) < 1e-4f)) return invalid("fg_hand_create: joint axes must be unit vectors");
    H.q_low[l - 1] = d->q_low[l - 1];
    H.q_up[l - 1] = d->q_up[l - 1];
    if (!(H.q_low[l - 1] <= H.q_up[l - 1])) return invalid("fg_hand_create: q_low must be <= q_up");
  }
  std::vector<float4> pts(P);
  int prev = 0;
  H.aligned32 = 1;
  for (int i = 0; i < P; ++i) {
    int l = d->link_of_point[i];
    if (l < 0 || l >= L || l < prev) return invalid("fg_hand_create: link_of_point must be nondecreasing in [0, L)");
    if (l != prev && (i & 31)) H.aligned32 = 0;
    prev = l;
    float x = d->pts_local[3 * i], y = d->pts_local[3 * i + 1], z = d->pts_local[3 * i + 2];
    if (!std::isfinite(x) || !std::isfinite(y) || !std::isfinite(z)) return invalid("fg_hand_create: non-finite point");
    pts[i] = make_float4(x, y, z, (float)l);
  }
  // bounding sphere (link frame) of every chunk of 32 consecutive points; a chunk
  // that spans two links is never culled (link -1)
  const int nchunks = (P + 31) / 32;
  H.nchunks = nchunks;
  std::vector<float4> spheres(nchunks);
  std::vector<int> clink(nchunks);
  for (int j = 0; j < nchunks; ++j) {
    const int b = 32 * j, e = std::min(P, b + 32);
    int l = d->link_of_point[b];
    for (int i = b; i < e; ++i)
      if (d->link_of_point[i] != l) l = -1;
    double c[3] = {0.0, 0.0, 0.0};
    for (int i = b; i < e; ++i)
      for (int k = 0; k < 3; ++k) c[k] += d->pts_local[3 * i + k];
    for (int k = 0; k < 3; ++k) c[k] /= (e - b);
    const float cf[3] = {(float)c[0], (float)c[1], (float)c[2]};
    double rad = 0.0;
    for (int i = b; i < e; ++i) {
      double r2 = 0.0;
      for (int k = 0; k < 3; ++k) {
        const double dk = (double)d->pts_local[3 * i + k] - (double)cf[k];
        r2 += dk * dk;
      }
      rad = std::max(rad, std::sqrt(r2));
    }
    spheres[j] = make_float4(cf[0], cf[1], cf[2], (float)(rad * (1.0 + 1e-6) + 1e-7));
    clink[j] = l;
  }
  // adjoint work units: each link's points in runs of at most kUnitPoints
  std::vector<int4> units;
  {
    int i = 0;
    for (int l = 0; l < L; ++l) {
      H.unit_begin[l] = (int)units.size();
      int e = i;
      while (e < P && d->link_of_point[e] == l) ++e;
      for (int b = i; b < e; b += kUnitPoints) units.push_back(make_int4(b, std::min(kUnitPoints, e - b), l, 0));
      i = e;
    }
    H.unit_begin[L] = (int)units.size();
    H.nunits = (int)units.size();
  }
  fg_hand* h = new (std::nothrow) fg_hand;
  if (!h) return FG_ERR_OOM;
  std::memset(h, 0, sizeof(*h));
  auto fail = [&](cudaError_t e, const char* what) {
    cudaFree(h->pts);
    cudaFree(h->chunk_sphere);
    cudaFree(h->chunk_link);
    cudaFree(h->units);
    cudaFree(h->dev);
    delete h;
    return cuda_status(e, what);
  };
  cudaError_t e = cudaMalloc(&h->pts, sizeof(float4) * P);
  if (e == cudaSuccess) e = cudaMalloc(&h->chunk_sphere, sizeof(float4) * nchunks);
  if (e == cudaSuccess) e = cudaMalloc(&h->chunk_link, sizeof(int) * nchunks);
  if (e == cudaSuccess) e = cudaMalloc(&h->units, sizeof(int4) * std::max<size_t>(units.size(), 1));
  if (e == cudaSuccess) e = cudaMalloc(&h->dev, sizeof(HandDev));
  if (e == cudaSuccess && alloc_fault()) e = cudaErrorMemoryAllocation;
  if (e != cudaSuccess) return fail(e, "fg_hand_create: cudaMalloc");
  H.pts = h->pts;
  H.chunk_sphere = h->chunk_sphere;
  H.chunk_link = h->chunk_link;
  H.units = h->units;
  e = cudaMemcpy(h->pts, pts.data(), sizeof(float4) * P, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->chunk_sphere, spheres.data(), sizeof(float4) * nchunks, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->chunk_link, clink.data(), sizeof(int) * nchunks, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !units.empty())
    e = cudaMemcpy(h->units, units.data(), sizeof(int4) * units.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->dev, &H, sizeof(HandDev), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(e, "fg_hand_create: cudaMemcpy");
  h->host = H;
  for (int l = 0; l < L; ++l) h->subtree_end[l] = H.subtree_end[l];
  *out = h;
  return FG_OK;
}

fg_status fg_hand_destroy(fg_hand* h) {
  if (!h) return FG_OK;
  cudaFree(h->pts);
  cudaFree(h->chunk_sphere);
  cudaFree(h->chunk_link);
  cudaFree(h->units);
  cudaFree(h->dev);
  delete h;
  return FG_OK;
}

fg_status fg_hand_info(const fg_hand* h, int* nl, int* nj, int* nd, int* np) {
  if (!h) return invalid("fg_hand_info: NULL hand");
  if (nl) *nl = h->host.L;
  if (nj) *nj = h->host.J;
  if (nd) *nd = h->host.D;
  if (np) *np = h->host.P;
  return FG_OK;
}

fg_status fg_sdf_create(const float* grid, int nx, int ny, int nz, const float* origin, float pitch, float mass,
                        float inertia, fg_sdf** out) {
  if (!grid || !origin || !out) return invalid("fg_sdf_create: NULL argument");
  *out = nullptr;
  if (nx < 2 || ny < 2 || nz < 2) return invalid("fg_sdf_create: grid dimensions must be >= 2");
  if ((double)nx * ny * nz > 2147483647.0) return invalid("fg_sdf_create: grid has more than 2^31 nodes");
  if (!(pitch > 0.0f) || !std::isfinite(pitch)) return invalid("fg_sdf_create: pitch must be > 0");
  if (!(mass > 0.0f) || !(inertia > 0.0f) || !std::isfinite(mass) || !std::isfinite(inertia))
    return invalid("fg_sdf_create: mass and inertia must be > 0");
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(origin[k])) return invalid("fg_sdf_create: non-finite origin");
  fg_sdf* s = new (std::nothrow) fg_sdf;
  if (!s) return FG_ERR_OOM;
  s->bytes = sizeof(float) * (size_t)nx * ny * nz;
  cudaError_t e = alloc_fault() ? cudaErrorMemoryAllocation : cudaMalloc(&s->grid, s->bytes);
  if (e != cudaSuccess) {
    delete s;
    return cuda_status(e, "fg_sdf_create: cudaMalloc");
  }
  e = cudaMemcpy(s->grid, grid, s->bytes, cudaMemcpyDefault);
  if (e != cudaSuccess) {
    cudaFree(s->grid);
    delete s;
    return cuda_status(e, "fg_sdf_create: cudaMemcpy");
  }
  ObjDev& o = s->host;
  std::memset(&o, 0, sizeof(o));
  o.grid = s->grid;
  o.nx = nx;
  o.ny = ny;
  o.nz = nz;
  o.ox = origin[0];
  o.oy = origin[1];
  o.oz = origin[2];
  o.h = pitch;
  o.inv_h = 1.0f / pitch;
  o.inv_mass = 1.0f / mass;
  o.inv_inertia = 1.0f / inertia;
  o.uo[0] = -origin[0] * o.inv_h;
  o.uo[1] = -origin[1] * o.inv_h;
  o.uo[2] = -origin[2] * o.inv_h;
  int levels = 0;
  const size_t pf = min_pyramid_floats(nx, ny, nz, &levels);
  s->pyr = nullptr;
  e = cudaMalloc(&s->pyr, sizeof(float) * pf);
  if (e == cudaSuccess) e = build_min_pyramid(s->grid, nx, ny, nz, s->pyr, levels, o.pyr_off);
  if (e != cudaSuccess) {
    cudaFree(s->pyr);
    cudaFree(s->grid);
    delete s;
    return cuda_status(e, "fg_sdf_create: min-pyramid");
  }
  o.pyr = s->pyr;
  o.pyr_levels = levels;
  o.kind = kObjGrid;
  s->pyr_bytes = sizeof(float) * pf;
  s->mesh = nullptr;
  *out = s;
  return FG_OK;
}

fg_status fg_sdf_destroy(fg_sdf* s) {
  if (!s) return FG_OK;
  cudaFree(s->mesh);
  cudaFree(s->pyr);
  cudaFree(s->grid);
  delete s;
  return FG_OK;
}

fg_status fg_scene_create(const fg_sdf* const* sdfs, int n, fg_scene** out) {
  if (!sdfs || !out || n < 1) return invalid("fg_scene_create: need n >= 1 objects");
  *out = nullptr;
  std::vector<ObjDev> tab(n);
  for (int i = 0; i < n; ++i) {
    if (!sdfs[i]) return invalid("fg_scene_create: NULL object");
    tab[i] = sdfs[i]->host;
  }
  fg_scene* sc = new (std::nothrow) fg_scene;
  if (!sc) return FG_ERR_OOM;
  sc->n = n;
  sc->has_mesh = 0;
  for (int i = 0; i < n; ++i) sc->has_mesh |= tab[i].kind == kObjMesh;
  cudaError_t e = cudaMalloc(&sc->dev, sizeof(ObjDev) * n);
  if (e != cudaSuccess) {
    delete sc;
    return cuda_status(e, "fg_scene_create: cudaMalloc");
  }
  e = cudaMemcpy(sc->dev, tab.data(), sizeof(ObjDev) * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(sc->dev);
    delete sc;
    return cuda_status(e, "fg_scene_create: cudaMemcpy");
  }
  *out = sc;
  return FG_OK;
}

fg_status fg_scene_destroy(fg_scene* sc) {
  if (!sc) return FG_OK;
  cudaFree(sc->dev);
  delete sc;
  return FG_OK;
}

fg_status fg_fk(const fg_hand* h, const float* q, int B, float* pts, void* stream) {
  if (!h) return invalid("fg_fk: NULL hand");
  if (B < 0) return invalid("fg_fk: B < 0");
  if (B == 0) return FG_OK;
  if (!q || !pts) return invalid("fg_fk: NULL buffer");
  if ((size_t)B * h->host.P > (size_t)1 << 40) return invalid("fg_fk: B * P too large");
  return cuda_status(launch_fk_points(h, q, B, pts, (cudaStream_t)stream), "fg_fk");
}

fg_status fg_sdf_query(const fg_sdf* s, const float* pts, int n, float r, float* phi, float* grad, void* stream) {
  if (!s) return invalid("fg_sdf_query: NULL sdf");
  if (n < 0) return invalid("fg_sdf_query: n < 0");
  if (n == 0) return FG_OK;
  if (!pts || !phi) return invalid("fg_sdf_query: NULL buffer");
  if (!std::isfinite(r)) return invalid("fg_sdf_query: non-finite r_dil");
  return cuda_status(launch_sdf_query(s->host, pts, n, r, phi, grad, (cudaStream_t)stream), "fg_sdf_query");
}

}  // extern "C"

namespace fg {

fg_status check_common(const char* fn, const fg_hand* h, const fg_scene* sc, int B, const fg_params* p) {
  if (!h || !sc) return invalid(std::string(fn) + ": NULL hand or scene");
  if (B < 0) return invalid(std::string(fn) + ": B < 0");
  return check_params(p);
}

// Entry points that implement the one-step metric only.
fg_status check_one_step(const char* fn, const fg_params* p) {
  if (p->sim_steps != 0)
    return invalid(std::string(fn) + ": params.sim_steps must be 0 here (T-step metric: fg_loss_and_grad, "
                   "fg_optimize_step)");
  if (p->gauss_seidel != 0)
    return invalid(std::string(fn) + ": params.gauss_seidel must be 0 here (Gauss-Seidel form: fg_loss_and_grad, "
                   "fg_optimize_step)");
  return FG_OK;
}

}  // namespace fg

extern "C" {

// The Gauss-Seidel form: hands whose chunks fit the kernel's tables.
static fg_status check_gs(const char* fn, const fg_hand* h, const fg_scene* sc) {
  (void)sc;
  if (h->host.nchunks > kMaxCullChunks)
    return invalid(std::string(fn) + ": the Gauss-Seidel form takes hands of at most 8,192 points");
  return FG_OK;
}

fg_status fg_contact_wrench(const fg_hand* h, const fg_scene* sc, const int* oc, const float* q, int B,
                            const fg_params* p, float r, float* wrench, int* ncontact, uint32_t* bits,
                            void* stream) {
  fg_status st = check_common("fg_contact_wrench", h, sc, B, p);
  if (st == FG_OK && p->sim_steps != 0)
    st = invalid("fg_contact_wrench: params.sim_steps must be 0 here (the T-step metric: fg_loss_and_grad, "
                 "fg_optimize_step)");
  if (st == FG_OK && p->gauss_seidel) st = check_gs("fg_contact_wrench", h, sc);
  if (st != FG_OK) return st;
  if (B == 0) return FG_OK;
  if (!q || !wrench || !ncontact) return invalid("fg_contact_wrench: NULL buffer");
  if (!std::isfinite(r)) return invalid("fg_contact_wrench: non-finite r_dil");
  FusedArgs a{};
  a.hand = h->dev;
  a.hand_D = h->host.D;
  a.objs = sc->dev;
  a.n_obj = sc->n;
  a.any_mesh = sc->has_mesh;
  a.obj_of_cand = oc;
  a.q = const_cast<float*>(q);
  a.B = B;
  a.P = params_from(p);
  a.r_fixed = r;
  a.nsteps = 1;
  a.wrench = wrench;
  a.ncontact = ncontact;
  a.bits = bits;
  if (a.P.gauss_seidel)
    return cuda_status(launch_gs(kModeWrench, a, h->host.nchunks, (cudaStream_t)stream),
                       "fg_contact_wrench (Gauss-Seidel)");
  return cuda_status(launch_fused(kModeWrench, a, h, (cudaStream_t)stream), "fg_contact_wrench");
}

fg_status fg_loss_and_grad(const fg_hand* h, const fg_scene* sc, const int* oc, const float* q, int B,
                           const fg_params* p, float r, float* loss, float* grad, void* stream) {
  fg_status st = check_common("fg_loss_and_grad", h, sc, B, p);
  if (st != FG_OK) return st;
  if (B == 0) return FG_OK;
  if (!q || !loss) return invalid("fg_loss_and_grad: NULL buffer");
  if (!std::isfinite(r)) return invalid("fg_loss_and_grad: non-finite r_dil");
  FusedArgs a{};
  a.hand = h->dev;
  a.hand_D = h->host.D;
  a.objs = sc->dev;
  a.n_obj = sc->n;
  a.any_mesh = sc->has_mesh;
  a.obj_of_cand = oc;
  a.q = const_cast<float*>(q);
  a.B = B;
  a.P = params_from(p);
  a.r_fixed = r;
  a.nsteps = 1;
  a.loss = loss;
  a.grad = grad;
  if (a.P.sim_steps >= 1) {
    return cuda_status(launch_tstep(kModeLossGrad, a, (cudaStream_t)stream), "fg_loss_and_grad (T-step)");
  }
  if (a.P.gauss_seidel) {
    st = check_gs("fg_loss_and_grad", h, sc);
    if (st != FG_OK) return st;
    return cuda_status(launch_gs(kModeLossGrad, a, h->host.nchunks, (cudaStream_t)stream),
                       "fg_loss_and_grad (Gauss-Seidel)");
  }
  return cuda_status(launch_fused(kModeLossGrad, a, h, (cudaStream_t)stream), "fg_loss_and_grad");
}

fg_status fg_optimize_step(const fg_hand* h, const fg_scene* sc, const int* oc, float* q, int B, const fg_params* p,
                           int step, int total_steps, int nsteps, float* loss, void* stream) {
  fg_status st = check_common("fg_optimize_step", h, sc, B, p);
  if (st != FG_OK) return st;
  if (nsteps < 1) return invalid("fg_optimize_step: nsteps must be >= 1");
  if (step < 0 || total_steps < 1) return invalid("fg_optimize_step: need step >= 0 and total_steps >= 1");
  if (B == 0) return FG_OK;
  if (!q) return invalid("fg_optimize_step: NULL q");
  FusedArgs a{};
  a.hand = h->dev;
  a.hand_D = h->host.D;
  a.objs = sc->dev;
  a.n_obj = sc->n;
  a.any_mesh = sc->has_mesh;
  a.obj_of_cand = oc;
  a.q = q;
  a.B = B;
  a.P = params_from(p);
  a.step0 = step;
  a.total_steps = total_steps;
  a.nsteps = nsteps;
  a.loss = loss;
  if (a.P.sim_steps >= 1) {
    return cuda_status(launch_tstep(kModeOptimize, a, (cudaStream_t)stream), "fg_optimize_step (T-step)");
  }
  if (a.P.gauss_seidel) {
    st = check_gs("fg_optimize_step", h, sc);
    if (st != FG_OK) return st;
    return cuda_status(launch_gs(kModeOptimize, a, h->host.nchunks, (cudaStream_t)stream),
                       "fg_optimize_step (Gauss-Seidel)");
  }
  return cuda_status(launch_fused(kModeOptimize, a, h, (cudaStream_t)stream), "fg_optimize_step");
}

fg_status fg_optimize_step_host(const fg_hand* h, const fg_scene* sc, const int* oc, const float* host_q_in,
                                float* q, int B, const fg_params* p, int step, int total_steps, int nsteps,
                                float* loss, float* host_q_out, float* host_loss, void* stream) {
  if (B > 0 && (!host_q_in || !q || !host_q_out)) return invalid("fg_optimize_step_host: NULL buffer");
  if (B > 0 && !h) return invalid("fg_optimize_step_host: NULL hand");
  if (host_loss && !loss) return invalid("fg_optimize_step_host: host_loss needs the device loss buffer");
  fg_status st = check_common("fg_optimize_step_host", h, sc, B, p);
  if (st != FG_OK) return st;
  if (B == 0) return FG_OK;
  const size_t qbytes = sizeof(float) * (size_t)B * h->host.D;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(q, host_q_in, qbytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_status(e, "fg_optimize_step_host (host to device)");
  st = fg_optimize_step(h, sc, oc, q, B, p, step, total_steps, nsteps, loss, stream);
  if (st != FG_OK) return st;
  e = cudaMemcpyAsync(host_q_out, q, qbytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && host_loss)
    e = cudaMemcpyAsync(host_loss, loss, sizeof(float) * (size_t)B, cudaMemcpyDeviceToHost, s);
  return cuda_status(e, "fg_optimize_step_host (device to host)");
}

fg_status fg_contact_measure(const fg_hand* h, const fg_scene* sc, const int* oc, const float* q, int B,
                             const float* weights, float tau, float* out, void* stream) {
  if (!h || !sc) return invalid("fg_contact_measure: NULL hand or scene");
  if (B < 0) return invalid("fg_contact_measure: B < 0");
  if (!std::isfinite(tau)) return invalid("fg_contact_measure: non-finite tau");
  if (B == 0) return FG_OK;
  if (!q || !weights || !out) return invalid("fg_contact_measure: NULL buffer");
  FusedArgs a{};
  a.hand = h->dev;
  a.hand_D = h->host.D;
  a.objs = sc->dev;
  a.n_obj = sc->n;
  a.any_mesh = sc->has_mesh;
  a.obj_of_cand = oc;
  a.q = const_cast<float*>(q);
  a.B = B;
  return cuda_status(launch_contact_measure(a, weights, tau, out, (cudaStream_t)stream), "fg_contact_measure");
}

fg_status fg_grasp_epsilon(const fg_hand* h, const fg_scene* sc, const int* oc, const float* q, int B, float tau,
                           float mu, int cone_edges, float torque_scale, const float* dirs, int K, float* eps,
                           int* n_contacts, void* stream) {
  if (!h || !sc) return invalid("fg_grasp_epsilon: NULL hand or scene");
  if (B < 0) return invalid("fg_grasp_epsilon: B < 0");
  if (!std::isfinite(tau)) return invalid("fg_grasp_epsilon: non-finite tau");
  if (!(mu >= 0.0f) || !std::isfinite(mu)) return invalid("fg_grasp_epsilon: mu must be >= 0");
  if (!(torque_scale >= 0.0f) || !std::isfinite(torque_scale))
    return invalid("fg_grasp_epsilon: torque_scale must be >= 0");
  if (cone_edges < 1 || cone_edges > 32) return invalid("fg_grasp_epsilon: cone_edges must be in [1, 32]");
  if (K < 1 || K > FG_MAX_DIRS) return invalid("fg_grasp_epsilon: K must be in [1, FG_MAX_DIRS]");
  if (B == 0) return FG_OK;
  if (!q || !dirs || !eps) return invalid("fg_grasp_epsilon: NULL buffer");
  FusedArgs a{};
  a.hand = h->dev;
  a.hand_D = h->host.D;
  a.objs = sc->dev;
  a.n_obj = sc->n;
  a.any_mesh = sc->has_mesh;
  a.obj_of_cand = oc;
  a.q = const_cast<float*>(q);
  a.B = B;
  return cuda_status(launch_grasp_epsilon(a, tau, mu, cone_edges, torque_scale, dirs, K, eps, n_contacts,
                                          (cudaStream_t)stream),
                     "fg_grasp_epsilon");
}

fg_status fg_plain_workspace_size(const fg_hand* h, int B, size_t* bytes) {
  if (!h || !bytes || B < 0) return invalid("fg_plain_workspace_size: bad argument");
  *bytes = plain_workspace_bytes(h, B);
  return FG_OK;
}

fg_status fg_optimize_step_plain(const fg_hand* h, const fg_scene* sc, const int* oc, float* q, int B,
                                 const fg_params* p, int step, int total_steps, int nsteps, float* loss, void* ws,
                                 size_t ws_bytes, void* stream) {
  fg_status st = check_common("fg_optimize_step_plain", h, sc, B, p);
  if (st == FG_OK) st = check_one_step("fg_optimize_step_plain", p);
  if (st != FG_OK) return st;
  if (sc->has_mesh) return invalid("fg_optimize_step_plain: the per-stage form takes grid objects only");
  if (nsteps < 1) return invalid("fg_optimize_step_plain: nsteps must be >= 1");
  if (step < 0 || total_steps < 1) return invalid("fg_optimize_step_plain: need step >= 0 and total_steps >= 1");
  if (B == 0) return FG_OK;
  if (!q || !ws) return invalid("fg_optimize_step_plain: NULL buffer");
  if (((uintptr_t)ws & 255) != 0) return invalid("fg_optimize_step_plain: workspace must be 256-byte aligned");
  if (ws_bytes < plain_workspace_bytes(h, B)) return invalid("fg_optimize_step_plain: workspace too small");
  return cuda_status(launch_plain_step(h, sc, oc, q, B, params_from(p), step, total_steps, nsteps, loss, ws,
                                       (cudaStream_t)stream),
                     "fg_optimize_step_plain");
}

fg_status fg_fused_config_count(int* n) {
  if (!n) return invalid("fg_fused_config_count: NULL");
  *n = fused_config_count();
  return FG_OK;
}

fg_status fg_fused_config_info(int index, int* nw, int* minb, int* ppt) {
  if (index < 0 || index >= fused_config_count() || !nw || !minb || !ppt)
    return invalid("fg_fused_config_info: bad index or NULL");
  fused_config_info(index, nw, minb, ppt);
  return FG_OK;
}

fg_status fg_fused_config_select(int index) {
  if (index < -1 || index >= fused_config_count()) return invalid("fg_fused_config_select: bad index");
  fused_config_select(index);
  return FG_OK;
}

fg_status fg_fused_config_current(int* index) {
  if (!index) return invalid("fg_fused_config_current: NULL");
  *index = fused_config_current();
  return FG_OK;
}

fg_status fg_autotune(const fg_hand* h, const fg_scene* sc, const int* oc, const float* q, int B, const fg_params* p,
                      int step, int total_steps, int nsteps, int reps, float* host_times_ms, int* best,
                      void* stream) {
  fg_status st = check_common("fg_autotune", h, sc, B, p);
  if (st == FG_OK) st = check_one_step("fg_autotune", p);
  if (st != FG_OK) return st;
  if (B < 1 || !q) return invalid("fg_autotune: need B >= 1 and q");
  if (nsteps < 1 || reps < 1 || step < 0 || total_steps < 1) return invalid("fg_autotune: bad step arguments");
  FusedArgs a{};
  a.hand = h->dev;
  a.hand_D = h->host.D;
  a.objs = sc->dev;
  a.n_obj = sc->n;
  a.any_mesh = sc->has_mesh;
  a.obj_of_cand = oc;
  a.q = const_cast<float*>(q);
  a.B = B;
  a.P = params_from(p);
  a.step0 = step;
  a.total_steps = total_steps;
  a.nsteps = nsteps;
  return cuda_status(autotune_fused(a, reps, host_times_ms, best, (cudaStream_t)stream), "fg_autotune");
}

}  // extern "C"
