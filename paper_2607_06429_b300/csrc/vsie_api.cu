// libvsie: handle lifetime, discretisation (create time) and the apply entry points.
//
// Create-time arithmetic follows the paper's definitions: alpha, beta (Eqs. alpha, beta),
// the mass function (Eq. mass_function), the weight (beta - k0^2 alpha) of the volume
// single layer, grad(alpha) of the volume adjoint double layer and the interface jump
// omega (alpha_1 on Gamma_1, alpha_2 - alpha_1 on Gamma_2) of the double layer, all from
// Eq. (vsie); P0 collocation at centroids (Sec. 2.3.4).  Per-element geometry is O(n)
// host work; the near-field/self correction matrix is built on the device.

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "vsie_internal.h"

namespace vsie {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }
void clear_error() { g_err.clear(); }

vsie_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "CUDA error %d (%s) in %s at %s:%d", (int)e,
           cudaGetErrorString(e), what, file, line);
  set_error(buf);
  cudaGetLastError();  // clear a non-sticky error
  return e == cudaErrorMemoryAllocation ? VSIE_ERR_OOM : VSIE_ERR_CUDA;
}

vsie_status dalloc(vsie_handle* h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    char buf[256];
    snprintf(buf, sizeof(buf), "device allocation of %zu bytes failed: %s", bytes,
             cudaGetErrorString(e));
    set_error(buf);
    cudaGetLastError();
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? VSIE_ERR_OOM : VSIE_ERR_CUDA;
  }
  h->allocs.push_back(*p);
  return VSIE_OK;
}

template <class T>
static vsie_status upload(vsie_handle* h, T** d, const std::vector<T>& v) {
  VSIE_TRY(dalloc_t(h, d, v.size()));
  if (!v.empty()) VSIE_CUDA(cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return VSIE_OK;
}

static inline bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// Degree-2 four-point rule on a tetrahedron: barycentric (a, b, b, b) and permutations,
// a = (5 + 3 sqrt5)/20, b = (5 - sqrt5)/20, weight |e|/4 each.
static void tet_points(const double* P /*4x3*/, double* out /*4x3*/) {
  const double s5 = std::sqrt(5.0);
  const double a = (5.0 + 3.0 * s5) / 20.0, b = (5.0 - s5) / 20.0;
  for (int q = 0; q < 4; ++q)
    for (int d = 0; d < 3; ++d) {
      double acc = 0.0;
      for (int v = 0; v < 4; ++v) acc += (v == q ? a : b) * P[3 * v + d];
      out[3 * q + d] = acc;
    }
}

// Degree-2 three-point interior rule on a triangle: barycentric (2/3, 1/6, 1/6).
static void tri_points(const double* P /*3x3*/, double* out /*3x3*/) {
  for (int q = 0; q < 3; ++q)
    for (int d = 0; d < 3; ++d) {
      double acc = 0.0;
      for (int v = 0; v < 3; ++v) acc += (v == q ? 2.0 / 3.0 : 1.0 / 6.0) * P[3 * v + d];
      out[3 * q + d] = acc;
    }
}

}  // namespace vsie

using namespace vsie;

extern "C" const char* vsie_last_error(void) { return g_err.c_str(); }

extern "C" void vsie_destroy(vsie_handle* h) {
  if (!h) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  for (void* p : h->allocs) cudaFree(p);
  if (h->gk_stream) cudaStreamDestroy(h->gk_stream);
  if (h->gk_fork) cudaEventDestroy(h->gk_fork);
  if (h->gk_join) cudaEventDestroy(h->gk_join);
  cudaSetDevice(prev);
  delete h;
}

extern "C" vsie_status vsie_sizes(const vsie_handle* h, int64_t* n, int64_t* n_far,
                                  int64_t* nnz) {
  if (!h) {
    set_error("vsie_sizes: null handle");
    return VSIE_ERR_ARG;
  }
  if (n) *n = h->n;
  if (n_far) *n_far = h->G.n + h->K.n + h->F.n;
  if (nnz) *nnz = h->C.nnz;
  return VSIE_OK;
}

// Per-element quantities of either mesh type, consumed by finish_create.
struct ElementGeometry {
  std::vector<double4_32a> tet_cen, tet_pts, tet_ga;   // volume elements ("tet" for either type)
  std::vector<double> tet_vol, tet_s, mass;
  std::vector<double4_32a> tri_vtx, tri_nrm, tri_cen, tri_pts;  // interface elements
  std::vector<double> tri_omega;
  int tri_npts = 3;  // far-rule points per interface element: 3 (triangles) or 1 (midpoint)
};

static vsie_status set_options(vsie_handle* h, const vsie_options* opt) {
  h->far_points = opt ? opt->tet_far_points : 1;
  h->near_radius = opt ? opt->near_radius : 0.0;
  h->tri_near_radius = opt ? opt->tri_near_radius : 0.0;
  h->tile_override = opt ? opt->tile_override : 0;
  h->debug_flags = opt ? opt->debug_flags : 0;
  if (h->far_points != 1 && h->far_points != 4) {
    set_error("vsie_create: tet_far_points must be 1 or 4");
    return VSIE_ERR_ARG;
  }
  if (!(h->near_radius >= 0.0) || !(h->tri_near_radius >= 0.0)) {
    set_error("vsie_create: negative near radius");
    return VSIE_ERR_ARG;
  }
  return VSIE_OK;
}

static vsie_status tet_geometry(const vsie_mesh* mesh, const vsie_material* mat, double k0, vsie_handle* h,
                                ElementGeometry& g) {
  const int64_t nv = mesh->n_vert, nt = mesh->n_tet, ns = mesh->n_tri;
  h->n_tet = nt;
  h->n_tri = ns;
  h->n = nt + ns;
  const double rho0 = mat->rho0, c0 = mat->c0;
  const double omega = k0 * c0;  // k0 = omega / c0
  auto& tet_cen = g.tet_cen;
  auto& tet_pts = g.tet_pts;
  auto& tet_ga = g.tet_ga;
  auto& tet_vol = g.tet_vol;
  auto& tet_s = g.tet_s;
  auto& mass = g.mass;
  auto& tri_vtx = g.tri_vtx;
  auto& tri_nrm = g.tri_nrm;
  auto& tri_cen = g.tri_cen;
  auto& tri_pts = g.tri_pts;
  auto& tri_omega = g.tri_omega;
  g.tri_npts = 3;
  // ---------------------------------------------------------------- volume elements
  tet_cen.resize(nt);
  tet_pts.resize(4 * nt);
  tet_ga.resize(nt);
  tet_vol.resize(nt);
  tet_s.resize(nt);
  mass.resize(h->n);
  for (int64_t e = 0; e < nt; ++e) {
    double P[12];
    for (int v = 0; v < 4; ++v) {
      int32_t id = mesh->tet[4 * e + v];
      if (id < 0 || id >= nv) {
        set_error("vsie_create: tetrahedron " + std::to_string(e) + " has a vertex index out of range");
        return VSIE_ERR_MESH;
      }
      for (int d = 0; d < 3; ++d) P[3 * v + d] = mesh->vert[3 * id + d];
    }
    const double d1[3] = {P[3] - P[0], P[4] - P[1], P[5] - P[2]};
    const double d2[3] = {P[6] - P[0], P[7] - P[1], P[8] - P[2]};
    const double d3[3] = {P[9] - P[0], P[10] - P[1], P[11] - P[2]};
    const double det = d1[0] * (d2[1] * d3[2] - d2[2] * d3[1]) -
                       d1[1] * (d2[0] * d3[2] - d2[2] * d3[0]) +
                       d1[2] * (d2[0] * d3[1] - d2[1] * d3[0]);
    const double vol = std::fabs(det) / 6.0;
    if (!(vol > 0.0) || !std::isfinite(vol)) {
      set_error("vsie_create: tetrahedron " + std::to_string(e) + " has zero volume");
      return VSIE_ERR_MESH;
    }
    const double rho = mat->rho[e], c = mat->c[e];
    if (!finite_pos(rho) || !finite_pos(c)) {
      set_error("vsie_create: non-positive or non-finite material on tetrahedron " + std::to_string(e));
      return VSIE_ERR_MESH;
    }
    const double alpha = rho0 / rho - 1.0;                                   // Eq. (alpha)
    const double beta = (rho0 / rho) * (omega / c) * (omega / c) - (omega / c0) * (omega / c0);  // Eq. (beta)
    tet_vol[e] = vol;
    tet_s[e] = beta - k0 * k0 * alpha;
    mass[e] = rho0 / rho;                                                   // Eq. (mass_function)
    tet_cen[e] = make_double4_32a(0.25 * (P[0] + P[3] + P[6] + P[9]), 0.25 * (P[1] + P[4] + P[7] + P[10]),
                              0.25 * (P[2] + P[5] + P[8] + P[11]), 0.0);
    double Q[12];
    tet_points(P, Q);
    for (int q = 0; q < 4; ++q) tet_pts[4 * e + q] = make_double4_32a(Q[3 * q], Q[3 * q + 1], Q[3 * q + 2], 0.0);
    if (mat->grad_alpha) {
      const double* g = mat->grad_alpha + 3 * e;
      if (!std::isfinite(g[0]) || !std::isfinite(g[1]) || !std::isfinite(g[2])) {
        set_error("vsie_create: non-finite grad_alpha");
        return VSIE_ERR_NAN;
      }
      tet_ga[e] = make_double4_32a(g[0], g[1], g[2], 0.0);
    } else {
      tet_ga[e] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    }
  }

  // ---------------------------------------------------------------- interface elements
  tri_vtx.resize(3 * ns);
  tri_nrm.resize(ns);
  tri_cen.resize(ns);
  tri_pts.resize(3 * ns);
  tri_omega.resize(ns);
  for (int64_t t = 0; t < ns; ++t) {
    double P[9];
    for (int v = 0; v < 3; ++v) {
      int32_t id = mesh->tri[3 * t + v];
      if (id < 0 || id >= nv) {
        set_error("vsie_create: triangle " + std::to_string(t) + " has a vertex index out of range");
        return VSIE_ERR_MESH;
      }
      for (int d = 0; d < 3; ++d) P[3 * v + d] = mesh->vert[3 * id + d];
      tri_vtx[3 * t + v] = make_double4_32a(P[3 * v], P[3 * v + 1], P[3 * v + 2], 0.0);
    }
    const double e1[3] = {P[3] - P[0], P[4] - P[1], P[5] - P[2]};
    const double e2[3] = {P[6] - P[0], P[7] - P[1], P[8] - P[2]};
    double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                    e1[0] * e2[1] - e1[1] * e2[0]};
    const double nn = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    if (!(nn > 0.0) || !std::isfinite(nn)) {
      set_error("vsie_create: triangle " + std::to_string(t) + " has zero area");
      return VSIE_ERR_MESH;
    }
    const double area = 0.5 * nn;
    tri_nrm[t] = make_double4_32a(cr[0] / nn, cr[1] / nn, cr[2] / nn, area);
    tri_cen[t] = make_double4_32a((P[0] + P[3] + P[6]) / 3.0, (P[1] + P[4] + P[7]) / 3.0,
                              (P[2] + P[5] + P[8]) / 3.0, 0.0);
    double Q[9];
    tri_points(P, Q);
    for (int q = 0; q < 3; ++q) tri_pts[3 * t + q] = make_double4_32a(Q[3 * q], Q[3 * q + 1], Q[3 * q + 2], 0.0);
    const double rin = mat->tri_rho_in[t], rout = mat->tri_rho_out[t];
    if (!finite_pos(rin) || !finite_pos(rout)) {
      set_error("vsie_create: non-positive interface density on triangle " + std::to_string(t));
      return VSIE_ERR_MESH;
    }
    // omega = alpha_in - alpha_out  (alpha_1 on Gamma_1, alpha_2 - alpha_1 on Gamma_2)
    tri_omega[t] = rho0 / rin - rho0 / rout;
    // m = (rho0/rho_in + rho0/rho_out)/2 (Eq. mass_function on Gamma_1 and Gamma_2)
    mass[nt + t] = 0.5 * (rho0 / rin + rho0 / rout);
  }

  return VSIE_OK;
}

// The faces of a cuboid grid across which the density jumps, in the unknown order: axis
// by axis (x, y, z), each in lattice order (face index along the axis first); outside the
// grid the exterior density rho0.  f(centre, axis, area, rho_in, rho_out) per face, "in"
// the cell below the face along its axis.
template <class F>
static void for_each_jump_face(const vsie_cuboid_grid* grid, const double* rho, double rho0, F&& f) {
  const int64_t N[3] = {grid->nx, grid->ny, grid->nz};
  const double* E[3] = {grid->x_edges, grid->y_edges, grid->z_edges};
  auto cell = [&](const int64_t* I) { return (I[0] * N[1] + I[1]) * N[2] + I[2]; };
  for (int ax = 0; ax < 3; ++ax) {
    const int b1 = (ax + 1) % 3, b2 = (ax + 2) % 3;  // the face's in-plane axes
    for (int64_t u = 0; u < (ax == 0 ? N[0] + 1 : N[0]); ++u)
      for (int64_t v = 0; v < (ax == 1 ? N[1] + 1 : N[1]); ++v)
        for (int64_t w = 0; w < (ax == 2 ? N[2] + 1 : N[2]); ++w) {
          const int64_t I[3] = {u, v, w};
          const int64_t a = I[ax];
          int64_t below[3] = {u, v, w};
          below[ax] = a - 1;
          const double rin = a > 0 ? rho[cell(below)] : rho0;
          const double rout = a < N[ax] ? rho[cell(I)] : rho0;
          if (rin == rout) continue;
          double ctr[3];
          ctr[ax] = E[ax][a];
          ctr[b1] = 0.5 * (E[b1][I[b1]] + E[b1][I[b1] + 1]);
          ctr[b2] = 0.5 * (E[b2][I[b2]] + E[b2][I[b2] + 1]);
          const double area = (E[b1][I[b1] + 1] - E[b1][I[b1]]) * (E[b2][I[b2] + 1] - E[b2][I[b2]]);
          f(ctr, ax, area, rin, rout);
        }
  }
}

// Cuboid grid (Sec. 2.3.4, computational domain and discrete representation): P0 unknowns
// on the cells and on the rectangular cell faces across which the density jumps; every
// integral by the midpoint rule (one far-field point per element), the single-layer self
// term over the ball of equal volume, the double-layer self term of a flat face 0, no near
// rules.  Cells in the order (i ny + j) nz + k; then the jump faces normal to x (face a
// between cells a-1 and a, the background outside the grid), ordered by (a, j, k), then
// those normal to y by (i, b, k), then those normal to z by (i, j, c); a face's normal is
// the +axis, "in" the cell below it and "out" the one above.
static vsie_status cuboid_geometry(const vsie_cuboid_grid* grid, const double* rho, const double* c,
                                   double k0, vsie_handle* h, ElementGeometry& g) {
  const int64_t nx = grid->nx, ny = grid->ny, nz = grid->nz;
  const double rho0 = h->rho0, c0 = h->c0;
  const double omega = k0 * c0;
  const double* E[3] = {grid->x_edges, grid->y_edges, grid->z_edges};
  const int64_t N[3] = {nx, ny, nz};
  for (int d = 0; d < 3; ++d)
    for (int64_t a = 0; a < N[d]; ++a)
      if (!(E[d][a + 1] > E[d][a]) || !std::isfinite(E[d][a]) || !std::isfinite(E[d][a + 1])) {
        set_error("vsie_create_cuboid: edge coordinates must be finite and strictly increasing");
        return VSIE_ERR_MESH;
      }
  const int64_t nc = nx * ny * nz;
  auto cell = [&](int64_t i, int64_t j, int64_t k) { return (i * ny + j) * nz + k; };
  g.tet_cen.resize(nc);
  g.tet_pts.resize(4 * nc);
  g.tet_ga.assign(nc, make_double4_32a(0.0, 0.0, 0.0, 0.0));
  g.tet_vol.resize(nc);
  g.tet_s.resize(nc);
  g.mass.resize(nc);
  for (int64_t i = 0; i < nx; ++i)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t k = 0; k < nz; ++k) {
        const int64_t e = cell(i, j, k);
        if (!finite_pos(rho[e]) || !finite_pos(c[e])) {
          set_error("vsie_create_cuboid: non-positive or non-finite material on cell " + std::to_string(e));
          return VSIE_ERR_MESH;
        }
        const double alpha = rho0 / rho[e] - 1.0;                                        // Eq. (alpha)
        const double beta = (rho0 / rho[e]) * (omega / c[e]) * (omega / c[e]) - (omega / c0) * (omega / c0);  // Eq. (beta)
        const double4_32a ctr = make_double4_32a(0.5 * (E[0][i] + E[0][i + 1]), 0.5 * (E[1][j] + E[1][j + 1]),
                                                 0.5 * (E[2][k] + E[2][k + 1]), 0.0);
        g.tet_cen[e] = ctr;
        for (int q = 0; q < 4; ++q) g.tet_pts[4 * e + q] = ctr;  // unused: no four-point rule
        g.tet_vol[e] = (E[0][i + 1] - E[0][i]) * (E[1][j + 1] - E[1][j]) * (E[2][k + 1] - E[2][k]);
        g.tet_s[e] = beta - k0 * k0 * alpha;
        g.mass[e] = rho0 / rho[e];                                                         // Eq. (mass_function)
      }
  // jump faces, axis by axis
  for_each_jump_face(grid, rho, rho0, [&](const double ctr[3], int ax, double area, double rin, double rout) {
    double nrm[3] = {0.0, 0.0, 0.0};
    nrm[ax] = 1.0;
    const double4_32a cc = make_double4_32a(ctr[0], ctr[1], ctr[2], 0.0);
    g.tri_cen.push_back(cc);
    for (int q = 0; q < 3; ++q) {  // unused: midpoint rule, no near rule
      g.tri_vtx.push_back(cc);
      g.tri_pts.push_back(cc);
    }
    g.tri_nrm.push_back(make_double4_32a(nrm[0], nrm[1], nrm[2], area));
    g.tri_omega.push_back(rho0 / rin - rho0 / rout);   // alpha_in - alpha_out
    g.mass.push_back(0.5 * (rho0 / rin + rho0 / rout));  // Eq. (mass_function) on an interface
  });
  g.tri_npts = 1;
  h->n_tet = nc;
  h->n_tri = (int64_t)g.tri_cen.size();
  h->n = h->n_tet + h->n_tri;
  if (h->n > (int64_t)INT32_MAX / 4) {
    set_error("vsie_create_cuboid: too many unknowns");
    return VSIE_ERR_ARG;
  }
  return VSIE_OK;
}

// Everything after the element geometry, common to both mesh types: far-field source
// classes, targets, records, and the self / near correction.
static vsie_status finish_create(vsie_handle* h, ElementGeometry& g) {
  const int64_t nt = h->n_tet, ns = h->n_tri;
  const double k0 = h->k0;
  const int FP = h->far_points;
  const auto& tet_cen = g.tet_cen;
  const auto& tet_pts = g.tet_pts;
  const auto& tet_ga = g.tet_ga;
  const auto& tet_vol = g.tet_vol;
  const auto& tet_s = g.tet_s;
  const auto& mass = g.mass;
  const auto& tri_vtx = g.tri_vtx;
  const auto& tri_nrm = g.tri_nrm;
  const auto& tri_cen = g.tri_cen;
  const auto& tri_pts = g.tri_pts;
  const auto& tri_omega = g.tri_omega;
  const int TP = g.tri_npts;
  // ---------------------------------------------------------------- far-field sources
  // G: volume points with grad(alpha) = 0; F: volume points with grad(alpha) != 0;
  // K: interface points (v = sigma n, sigma = -omega w since dG/dn_y = -grad_x G . n).
  std::vector<double4_32a> g_ps, f_ps, f_v, k_ps, k_v, k_aux;
  std::vector<int32_t> g_own, f_own, k_own, g_first, g_elem, f_first, f_elem, k_first, k_elem;
  for (int64_t e = 0; e < nt; ++e) {
    const bool has_v = tet_ga[e].x != 0.0 || tet_ga[e].y != 0.0 || tet_ga[e].z != 0.0;
    auto& ps = has_v ? f_ps : g_ps;
    auto& own = has_v ? f_own : g_own;
    auto& first = has_v ? f_first : g_first;
    auto& el = has_v ? f_elem : g_elem;
    first.push_back((int32_t)ps.size());
    el.push_back((int32_t)e);
    const int npts = FP == 1 ? 1 : 4;
    const double w = tet_vol[e] / npts;
    for (int q = 0; q < npts; ++q) {
      const double4_32a y = FP == 1 ? tet_cen[e] : tet_pts[4 * e + q];
      ps.push_back(make_double4_32a(y.x, y.y, y.z, tet_s[e] * w));
      own.push_back((int32_t)e);
      if (has_v) f_v.push_back(make_double4_32a(tet_ga[e].x * w, tet_ga[e].y * w, tet_ga[e].z * w, 0.0));
    }
  }
  for (int64_t t = 0; t < ns; ++t) {
    k_first.push_back((int32_t)k_ps.size());
    k_elem.push_back((int32_t)(nt + t));
    const double w = tri_nrm[t].w / TP;
    const double sigma = -tri_omega[t] * w;
    for (int q = 0; q < TP; ++q) {
      const double4_32a y = TP == 1 ? tri_cen[t] : tri_pts[3 * t + q];
      k_ps.push_back(make_double4_32a(y.x, y.y, y.z, 0.0));
      k_v.push_back(make_double4_32a(sigma * tri_nrm[t].x, sigma * tri_nrm[t].y, sigma * tri_nrm[t].z, 0.0));
      k_aux.push_back(make_double4_32a(tri_nrm[t].x, tri_nrm[t].y, tri_nrm[t].z, sigma));
      k_own.push_back((int32_t)(nt + t));
    }
  }
  g_first.push_back((int32_t)g_ps.size());
  f_first.push_back((int32_t)f_ps.size());
  k_first.push_back((int32_t)k_ps.size());

  // ---------------------------------------------------------------- targets
  std::vector<double4_32a> tgt(h->n);
  std::vector<float4> tgt32(h->n);
  for (int64_t e = 0; e < nt; ++e) tgt[e] = tet_cen[e];
  for (int64_t t = 0; t < ns; ++t) tgt[nt + t] = tri_cen[t];
  const double kap = k0 / (2.0 * kPi);  // positions in units of the wavelength
  for (int64_t i = 0; i < h->n; ++i)
    tgt32[i] = make_float4((float)(kap * tgt[i].x), (float)(kap * tgt[i].y), (float)(kap * tgt[i].z), 0.0f);

  // double-float copies of kappa x for the precision-48 sums: (hi x3, 0) (lo x3, 0)
  std::vector<float4> tgtdf(2 * (size_t)h->n);
  for (int64_t i = 0; i < h->n; ++i) {
    const double v[3] = {kap * tgt[i].x, kap * tgt[i].y, kap * tgt[i].z};
    float hi[3], lo[3];
    for (int d = 0; d < 3; ++d) {
      hi[d] = (float)v[d];
      lo[d] = (float)(v[d] - (double)hi[d]);
    }
    tgtdf[2 * i] = make_float4(hi[0], hi[1], hi[2], 0.0f);
    tgtdf[2 * i + 1] = make_float4(lo[0], lo[1], lo[2], 0.0f);
  }
  VSIE_TRY(upload(h, &h->tgt64, tgt));
  VSIE_TRY(upload(h, &h->tgt32, tgt32));
  VSIE_TRY(upload(h, &h->tgtdf, tgtdf));
  VSIE_TRY(upload(h, &h->mass, mass));

  auto setup_class = [&](Sources& S, const std::vector<double4_32a>& ps, const std::vector<double4_32a>* vv,
                         const std::vector<double4_32a>* aux, const std::vector<int32_t>& own,
                         const std::vector<int32_t>& first, const std::vector<int32_t>& el,
                         int recs) -> vsie_status {
    S.n = (int64_t)ps.size();
    S.n_elem = (int64_t)el.size();
    VSIE_TRY(upload(h, &S.pos_s, ps));
    if (vv) VSIE_TRY(upload(h, &S.vvec, *vv));
    if (aux) VSIE_TRY(upload(h, &S.aux, *aux));
    VSIE_TRY(upload(h, &S.owner, own));
    VSIE_TRY(upload(h, &S.elem_first, first));
    VSIE_TRY(upload(h, &S.elem_list, el));
    VSIE_TRY(dalloc_t(h, &S.r32a, (size_t)recs * S.n));
    VSIE_TRY(dalloc_t(h, &S.r64a, (size_t)recs * S.n));
    if (recs == 1) {
      VSIE_TRY(dalloc_t(h, &S.r32b, (size_t)S.n));
      VSIE_TRY(dalloc_t(h, &S.r64b, (size_t)S.n));
    }
    VSIE_TRY(dalloc_t(h, &S.rdf, (size_t)(recs == 1 ? 3 : recs == 2 ? 4 : 6) * S.n));
    return VSIE_OK;
  };
  VSIE_TRY(setup_class(h->G, g_ps, nullptr, nullptr, g_own, g_first, g_elem, 1));
  VSIE_TRY(setup_class(h->K, k_ps, &k_v, &k_aux, k_own, k_first, k_elem, 2));
  VSIE_TRY(setup_class(h->F, f_ps, &f_v, nullptr, f_own, f_first, f_elem, 3));

  // ---------------------------------------------------------------- correction matrix
  double4_32a *d_tet_cen, *d_tet_pts, *d_tet_ga, *d_tri_vtx, *d_tri_nrm, *d_tri_pts, *d_tri_cen;
  double *d_tet_s, *d_tet_vol, *d_tri_omega;
  VSIE_TRY(upload(h, &d_tet_cen, tet_cen));
  VSIE_TRY(upload(h, &d_tet_pts, tet_pts));
  VSIE_TRY(upload(h, &d_tet_ga, tet_ga));
  VSIE_TRY(upload(h, &d_tet_s, tet_s));
  VSIE_TRY(upload(h, &d_tet_vol, tet_vol));
  VSIE_TRY(upload(h, &d_tri_vtx, tri_vtx));
  VSIE_TRY(upload(h, &d_tri_nrm, tri_nrm));
  VSIE_TRY(upload(h, &d_tri_omega, tri_omega));
  VSIE_TRY(upload(h, &d_tri_pts, tri_pts));
  VSIE_TRY(upload(h, &d_tri_cen, tri_cen));
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t i = 0; i < h->n; ++i) {
    const double p[3] = {tgt[i].x, tgt[i].y, tgt[i].z};
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::fmin(lo[d], p[d]);
      hi[d] = std::fmax(hi[d], p[d]);
    }
  }
  VSIE_TRY(build_correction(h, d_tet_cen, d_tet_pts, d_tet_s, d_tet_ga, d_tet_vol, d_tri_vtx,
                            d_tri_pts, d_tri_cen, d_tri_nrm, d_tri_omega, lo, hi));
  // the geometry stays with the handle: field evaluation at arbitrary points builds its
  // near-rule rows from it (about 200 bytes per tetrahedron)
  VSIE_CUDA(cudaDeviceSynchronize());
  noalloc_prepare(h->device);
  return VSIE_OK;
}

static vsie_status create_impl(const vsie_mesh* mesh, const vsie_material* mat, double k0,
                               const vsie_options* opt, vsie_handle* h) {
  h->k0 = k0;
  h->rho0 = mat->rho0;
  h->c0 = mat->c0;
  VSIE_TRY(set_options(h, opt));
  ElementGeometry g;
  VSIE_TRY(tet_geometry(mesh, mat, k0, h, g));
  return finish_create(h, g);
}

extern "C" vsie_status vsie_create(const vsie_mesh* mesh, const vsie_material* mat, double k0,
                                   const vsie_options* opt, vsie_handle** out) {
  clear_error();
  TraceRange trace("vsie_create");
  if (!out) {
    set_error("vsie_create: null output pointer");
    return VSIE_ERR_ARG;
  }
  *out = nullptr;
  if (!mesh || !mat || !mesh->vert || (mesh->n_tet > 0 && !mesh->tet) ||
      (mesh->n_tri > 0 && (!mesh->tri || !mat->tri_rho_in || !mat->tri_rho_out)) ||
      (mesh->n_tet > 0 && (!mat->rho || !mat->c))) {
    set_error("vsie_create: null mesh or material array");
    return VSIE_ERR_ARG;
  }
  if (mesh->n_vert <= 0 || mesh->n_tet < 0 || mesh->n_tri < 0 || mesh->n_tet + mesh->n_tri <= 0 ||
      mesh->n_tet + mesh->n_tri > (int64_t)INT32_MAX / 4) {
    set_error("vsie_create: mesh sizes out of range");
    return VSIE_ERR_ARG;
  }
  if (!(k0 > 0.0) || !std::isfinite(k0) || !finite_pos(mat->rho0) || !finite_pos(mat->c0)) {
    set_error("vsie_create: k0, rho0 and c0 must be positive and finite");
    return VSIE_ERR_ARG;
  }
  vsie_handle* h = new vsie_handle();
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__);
  }
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  vsie_status s = create_impl(mesh, mat, k0, opt, h);
  if (s != VSIE_OK) {
    std::string msg = vsie_last_error();
    vsie_destroy(h);
    set_error(msg);
    return s;
  }
  auto& in = h->inputs;
  in.kind = 0;
  in.vert.assign(mesh->vert, mesh->vert + 3 * mesh->n_vert);
  in.tet.assign(mesh->tet, mesh->tet + 4 * mesh->n_tet);
  if (mesh->n_tri) {
    in.tri.assign(mesh->tri, mesh->tri + 3 * mesh->n_tri);
    in.tri_rho_in.assign(mat->tri_rho_in, mat->tri_rho_in + mesh->n_tri);
    in.tri_rho_out.assign(mat->tri_rho_out, mat->tri_rho_out + mesh->n_tri);
  }
  if (mesh->n_tet) {
    in.rho.assign(mat->rho, mat->rho + mesh->n_tet);
    in.c.assign(mat->c, mat->c + mesh->n_tet);
  }
  in.has_grad_alpha = mat->grad_alpha != nullptr;
  if (in.has_grad_alpha) in.grad_alpha.assign(mat->grad_alpha, mat->grad_alpha + 3 * mesh->n_tet);
  in.has_opt = opt != nullptr;
  if (opt) in.opt = *opt;
  *out = h;
  return VSIE_OK;
}

// Rebuild every frequency-dependent part of the handle (weights, records, correction) for
// a new k0 from the saved creation inputs; the material, geometry and autotuned shapes stay.
extern "C" vsie_status vsie_set_frequency(vsie_handle* h, double k0) {
  clear_error();
  TraceRange trace("vsie_set_frequency");
  if (!h || !(k0 > 0.0) || !std::isfinite(k0)) {
    set_error("vsie_set_frequency: null handle or k0 not positive and finite");
    return VSIE_ERR_ARG;
  }
  VSIE_CUDA(cudaDeviceSynchronize());
  const int device = h->device, sms = h->num_sms;
  const double rho0 = h->rho0, c0 = h->c0;
  const auto tune = h->tune;
  auto inputs = std::move(h->inputs);
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  *h = vsie_handle();
  h->device = device;
  h->num_sms = sms;
  h->tune = tune;
  h->inputs = std::move(inputs);
  auto& in = h->inputs;
  vsie_status s;
  if (in.kind == 0) {
    const vsie_mesh mesh{(int64_t)(in.vert.size() / 3), in.vert.data(), (int64_t)(in.tet.size() / 4),
                         in.tet.data(), (int64_t)(in.tri.size() / 3), in.tri.empty() ? nullptr : in.tri.data()};
    const vsie_material mat{rho0, c0, in.rho.data(), in.c.data(),
                            in.has_grad_alpha ? in.grad_alpha.data() : nullptr,
                            in.tri_rho_in.empty() ? nullptr : in.tri_rho_in.data(),
                            in.tri_rho_out.empty() ? nullptr : in.tri_rho_out.data()};
    s = create_impl(&mesh, &mat, k0, in.has_opt ? &in.opt : nullptr, h);
  } else {
    const vsie_cuboid_grid grid{(int32_t)in.x_edges.size() - 1, (int32_t)in.y_edges.size() - 1,
                                (int32_t)in.z_edges.size() - 1, in.x_edges.data(), in.y_edges.data(),
                                in.z_edges.data()};
    h->k0 = k0;
    h->rho0 = rho0;
    h->c0 = c0;
    vsie_options opt{};
    opt.tet_far_points = 1;
    ElementGeometry g;
    s = set_options(h, &opt);
    if (s == VSIE_OK) s = cuboid_geometry(&grid, in.rho.data(), in.c.data(), k0, h, g);
    if (s == VSIE_OK) s = finish_create(h, g);
  }
  if (s != VSIE_OK) {
    // leave an empty operator (n = 0, no buffers): every call on it is a no-op or an
    // argument error, and a later vsie_set_frequency may rebuild it
    const std::string msg = vsie_last_error();
    cudaDeviceSynchronize();
    for (void* p : h->allocs) cudaFree(p);
    h->allocs.clear();
    auto keep = std::move(h->inputs);
    *h = vsie_handle();
    h->device = device;
    h->num_sms = sms;
    h->tune = tune;
    h->rho0 = rho0;
    h->c0 = c0;
    h->inputs = std::move(keep);
    set_error(msg);
  }
  return s;
}

// Host-only description of the interface unknowns of a cuboid grid (the faces in their
// unknown order), for callers that map solution vectors back to the grid.
extern "C" vsie_status vsie_cuboid_faces(const vsie_cuboid_grid* grid, const double* rho, double rho0,
                                         int64_t capacity, int64_t* n_faces, double* centres, int32_t* axis,
                                         double* area, double* omega, double* mass) {
  clear_error();
  if (!grid || !rho || !n_faces || !grid->x_edges || !grid->y_edges || !grid->z_edges || grid->nx < 1 ||
      grid->ny < 1 || grid->nz < 1 || capacity < 0 || !finite_pos(rho0)) {
    set_error("vsie_cuboid_faces: invalid argument");
    return VSIE_ERR_ARG;
  }
  const double* E[3] = {grid->x_edges, grid->y_edges, grid->z_edges};
  const int64_t N[3] = {grid->nx, grid->ny, grid->nz};
  for (int d = 0; d < 3; ++d)
    for (int64_t a = 0; a < N[d]; ++a)
      if (!(E[d][a + 1] > E[d][a]) || !std::isfinite(E[d][a]) || !std::isfinite(E[d][a + 1])) {
        set_error("vsie_cuboid_faces: edge coordinates must be finite and strictly increasing");
        return VSIE_ERR_MESH;
      }
  for (int64_t e = 0; e < N[0] * N[1] * N[2]; ++e)
    if (!finite_pos(rho[e])) {
      set_error("vsie_cuboid_faces: non-positive or non-finite density on cell " + std::to_string(e));
      return VSIE_ERR_MESH;
    }
  int64_t count = 0;
  for_each_jump_face(grid, rho, rho0, [&](const double ctr[3], int ax, double a, double rin, double rout) {
    if (count < capacity) {
      if (centres)
        for (int d = 0; d < 3; ++d) centres[3 * count + d] = ctr[d];
      if (axis) axis[count] = ax;
      if (area) area[count] = a;
      if (omega) omega[count] = rho0 / rin - rho0 / rout;
      if (mass) mass[count] = 0.5 * (rho0 / rin + rho0 / rout);
    }
    ++count;
  });
  *n_faces = count;
  if (count > capacity && (centres || axis || area || omega || mass)) {
    set_error("vsie_cuboid_faces: capacity smaller than the number of faces");
    return VSIE_ERR_ARG;
  }
  return VSIE_OK;
}

extern "C" vsie_status vsie_create_cuboid(const vsie_cuboid_grid* grid, const double* rho, const double* c,
                                          double rho0, double c0, double k0, vsie_handle** out) {
  clear_error();
  TraceRange trace("vsie_create_cuboid");
  if (!out) {
    set_error("vsie_create_cuboid: null output pointer");
    return VSIE_ERR_ARG;
  }
  *out = nullptr;
  if (!grid || !rho || !c || !grid->x_edges || !grid->y_edges || !grid->z_edges) {
    set_error("vsie_create_cuboid: null grid or material array");
    return VSIE_ERR_ARG;
  }
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 ||
      (int64_t)grid->nx * grid->ny * grid->nz > (int64_t)INT32_MAX / 8) {
    set_error("vsie_create_cuboid: grid sizes out of range");
    return VSIE_ERR_ARG;
  }
  if (!(k0 > 0.0) || !std::isfinite(k0) || !finite_pos(rho0) || !finite_pos(c0)) {
    set_error("vsie_create_cuboid: k0, rho0 and c0 must be positive and finite");
    return VSIE_ERR_ARG;
  }
  vsie_handle* h = new vsie_handle();
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__);
  }
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  h->k0 = k0;
  h->rho0 = rho0;
  h->c0 = c0;
  vsie_options opt{};
  opt.tet_far_points = 1;  // midpoint rule, no near rules
  ElementGeometry g;
  vsie_status s = set_options(h, &opt);
  if (s == VSIE_OK) s = cuboid_geometry(grid, rho, c, k0, h, g);
  if (s == VSIE_OK) s = finish_create(h, g);
  if (s != VSIE_OK) {
    std::string msg = vsie_last_error();
    vsie_destroy(h);
    set_error(msg);
    return s;
  }
  auto& in = h->inputs;
  in.kind = 1;
  in.x_edges.assign(grid->x_edges, grid->x_edges + grid->nx + 1);
  in.y_edges.assign(grid->y_edges, grid->y_edges + grid->ny + 1);
  in.z_edges.assign(grid->z_edges, grid->z_edges + grid->nz + 1);
  const size_t ncell = (size_t)grid->nx * grid->ny * grid->nz;
  in.rho.assign(rho, rho + ncell);
  in.c.assign(c, c + ncell);
  *out = h;
  return VSIE_OK;
}

namespace vsie {
vsie_status apply_one(vsie_handle* h, const double2* x, double2* y, int precision,
                      cudaStream_t st) {
  VSIE_TRY(far_apply(h, x, y, precision, st));
  VSIE_TRY(correction_apply(h, x, y, precision, st));
  return VSIE_OK;
}
}  // namespace vsie

static vsie_status check_apply_args(vsie_handle* h, const void* x, const void* y, int32_t nrhs,
                                    int32_t precision, const char* who) {
  if (!h || !x || !y) {
    set_error(std::string(who) + ": null handle or vector");
    return VSIE_ERR_ARG;
  }
  if (nrhs < 1) {
    set_error(std::string(who) + ": nrhs must be >= 1");
    return VSIE_ERR_ARG;
  }
  if (precision != 32 && precision != 48 && precision != 64) {
    set_error(std::string(who) + ": precision must be 32, 48 or 64");
    return VSIE_ERR_ARG;
  }
  if (x == y) {
    set_error(std::string(who) + ": input and output must not alias");
    return VSIE_ERR_ARG;
  }
  return VSIE_OK;
}

extern "C" vsie_status vsie_apply(vsie_handle* h, const void* d_x, void* d_y, int32_t nrhs,
                                  int32_t precision, void* stream) {
  clear_error();
  TraceRange trace("vsie_apply");
  VSIE_TRY(check_apply_args(h, d_x, d_y, nrhs, precision, "vsie_apply"));
  cudaStream_t st = (cudaStream_t)stream;
  const double2* x = (const double2*)d_x;
  double2* y = (double2*)d_y;
  for (int r = 0; r < nrhs; ++r)
    VSIE_TRY(apply_one(h, x + (size_t)r * h->n, y + (size_t)r * h->n, precision, st));
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

extern "C" vsie_status vsie_apply_rows(vsie_handle* h, const void* d_x, void* d_y, int64_t row_begin,
                                       int64_t row_end, int32_t precision, void* stream) {
  clear_error();
  TraceRange trace("vsie_apply_rows");
  VSIE_TRY(check_apply_args(h, d_x, d_y, 1, precision, "vsie_apply_rows"));
  if (row_begin < 0 || row_end < row_begin || row_end > h->n) {
    set_error("vsie_apply_rows: rows must satisfy 0 <= row_begin <= row_end <= n (n = " +
              std::to_string(h->n) + ")");
    return VSIE_ERR_ARG;
  }
  const int64_t m = row_end - row_begin;
  if (m == 0) return VSIE_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const double2* x = (const double2*)d_x;
  double2* y = (double2*)d_y;
  // the far sums of vsie_apply with the collocation records of the rows as targets (they
  // zero y first), then the rows' correction and mass
  VSIE_TRY(far_sums_at(h, x, h->tgt64 + row_begin, h->tgt32 + row_begin, h->tgtdf + 2 * row_begin, m, y,
                       precision, st));
  VSIE_TRY(correction_apply_rows(h, x, y, row_begin, row_end, precision, st));
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

extern "C" vsie_status vsie_apply_host(vsie_handle* h, const double* h_x, double* h_y,
                                       int32_t nrhs, int32_t precision, void* stream) {
  clear_error();
  TraceRange trace("vsie_apply_host");
  VSIE_TRY(check_apply_args(h, h_x, h_y, nrhs, precision, "vsie_apply_host"));
  cudaStream_t st = (cudaStream_t)stream;
  if (h->host_cols < nrhs) {
    VSIE_TRY(dalloc_t(h, &h->host_x, (size_t)h->n * nrhs));
    VSIE_TRY(dalloc_t(h, &h->host_y, (size_t)h->n * nrhs));
    h->host_cols = nrhs;
  }
  const size_t bytes = sizeof(double2) * (size_t)h->n * nrhs;
  VSIE_CUDA(cudaMemcpyAsync(h->host_x, h_x, bytes, cudaMemcpyHostToDevice, st));
  for (int r = 0; r < nrhs; ++r)
    VSIE_TRY(apply_one(h, h->host_x + (size_t)r * h->n, h->host_y + (size_t)r * h->n, precision, st));
  VSIE_CUDA(cudaMemcpyAsync(h_y, h->host_y, bytes, cudaMemcpyDeviceToHost, st));
  VSIE_CUDA(cudaStreamSynchronize(st));
  return VSIE_OK;
}

extern "C" vsie_status vsie_adjoint_apply(vsie_handle* h, const void* d_y, void* d_x,
                                          int32_t nrhs, int32_t precision, void* stream) {
  clear_error();
  TraceRange trace("vsie_adjoint_apply");
  VSIE_TRY(check_apply_args(h, d_y, d_x, nrhs, precision, "vsie_adjoint_apply"));
  if (precision == 48) {
    set_error("vsie_adjoint_apply: precision must be 32 or 64");
    return VSIE_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const double2* lam = (const double2*)d_y;
  double2* x = (double2*)d_x;
  for (int r = 0; r < nrhs; ++r) {
    VSIE_TRY(far_adjoint(h, lam + (size_t)r * h->n, x + (size_t)r * h->n, precision, st));
    VSIE_TRY(correction_adjoint(h, lam + (size_t)r * h->n, x + (size_t)r * h->n, precision, st));
  }
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

extern "C" vsie_status vsie_apply_timed(vsie_handle* h, const void* d_x, void* d_y,
                                        int32_t precision, void* stream, double* kernel_ms,
                                        int32_t* launches) {
  clear_error();
  TraceRange trace("vsie_apply_timed");
  VSIE_TRY(check_apply_args(h, d_x, d_y, 1, precision, "vsie_apply_timed"));
  if (!kernel_ms) {
    set_error("vsie_apply_timed: null kernel_ms");
    return VSIE_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const double2* x = (const double2*)d_x;
  double2* y = (double2*)d_y;
  cudaEvent_t ev[5];
  for (int i = 0; i < 5; ++i) VSIE_CUDA(cudaEventCreate(&ev[i]));
  int n_launch = 0;
  vsie_status s = VSIE_OK;
  auto run = [&]() -> vsie_status {
    VSIE_CUDA(cudaEventRecord(ev[0], st));
    VSIE_TRY(far_prescale(h, x, precision, st, &n_launch));
    VSIE_CUDA(cudaEventRecord(ev[1], st));
    VSIE_TRY(far_sum_g(h, y, precision, st, &n_launch));
    VSIE_CUDA(cudaEventRecord(ev[2], st));
    VSIE_TRY(far_sum_f(h, y, precision, st, &n_launch));
    VSIE_CUDA(cudaEventRecord(ev[3], st));
    VSIE_TRY(correction_apply(h, x, y, precision, st));
    n_launch += (h->n > 0) ? 2 : 0;  // x to double-float, then the CSR correction + mass
    n_launch += far_gk_extra_launches(h, precision);
    VSIE_CUDA(cudaEventRecord(ev[4], st));
    VSIE_CUDA(cudaEventSynchronize(ev[4]));
    for (int i = 0; i < 4; ++i) {
      float ms = 0.0f;
      VSIE_CUDA(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
      kernel_ms[i] = ms;
    }
    return VSIE_OK;
  };
  s = run();
  for (int i = 0; i < 5; ++i) cudaEventDestroy(ev[i]);
  if (launches) *launches = n_launch;
  return s;
}

extern "C" vsie_status vsie_apply_batched(vsie_handle* h, const void* d_x, void* d_y, int32_t nrhs,
                                          int32_t precision, void* stream) {
  clear_error();
  TraceRange trace("vsie_apply_batched");
  VSIE_TRY(check_apply_args(h, d_x, d_y, nrhs, precision, "vsie_apply_batched"));
  if (precision == 48) {
    set_error("vsie_apply_batched: precision must be 32 or 64");
    return VSIE_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const double2* x = (const double2*)d_x;
  double2* y = (double2*)d_y;
  if (precision == 32) {
    VSIE_TRY(apply_batched_multi_launch(&h, 1, &x, &y, nrhs, st));
    return batch_status(h, st);
  }
  VSIE_TRY(far_batched64_gk(h, x, y, nrhs, st));
  if (h->F.n)
    for (int r = 0; r < nrhs; ++r)
      VSIE_TRY(far_sum_f_only(h, x + (size_t)r * h->n, y + (size_t)r * h->n, 64, st));
  VSIE_TRY(correction_apply_block(h, x, y, nrhs, 64, st));
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

namespace vsie {

vsie_status check_multi_args(vsie_handle* const* hs, int32_t nop, const void* const* x, void* const* y,
                             int32_t nrhs, const char* who) {
  if (!hs || !x || !y || nop < 1 || nrhs < 1) {
    set_error(std::string(who) + ": null array, nop < 1 or nrhs < 1");
    return VSIE_ERR_ARG;
  }
  for (int p = 0; p < nop; ++p) {
    if (!hs[p] || !x[p] || !y[p] || x[p] == y[p]) {
      set_error(std::string(who) + ": null handle or vector, or input aliasing output");
      return VSIE_ERR_ARG;
    }
    const vsie_handle* a = hs[0];
    const vsie_handle* b = hs[p];
    if (b->n != a->n || b->G.n != a->G.n || b->K.n != a->K.n || b->F.n != a->F.n || b->device != a->device) {
      set_error(std::string(who) + ": operators differ in size (collocation points or far-field "
                "sources per class) or device");
      return VSIE_ERR_ARG;
    }
    for (int q = 0; q < p; ++q)
      if (hs[q] == hs[p]) {
        set_error(std::string(who) + ": an operator appears twice (its scratch buffers would be shared)");
        return VSIE_ERR_ARG;
      }
  }
  return VSIE_OK;
}

vsie_status apply_batched_multi_launch(vsie_handle* const* hs, int nop, const double2* const* x,
                                       double2* const* y, int nrhs, cudaStream_t st) {
  VSIE_TRY(far_batched_gk_multi(hs, nop, x, y, nrhs, st));
  for (int p = 0; p < nop; ++p) {
    vsie_handle* h = hs[p];
    if (h->F.n)
      for (int r = 0; r < nrhs; ++r)
        VSIE_TRY(far_sum_f_only(h, x[p] + (size_t)r * h->n, y[p] + (size_t)r * h->n, 32, st));
    VSIE_TRY(correction_apply_block(h, x[p], y[p], nrhs, 32, st));
  }
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

}  // namespace vsie

extern "C" vsie_status vsie_gradient_channels(vsie_handle* h, const void* d_lam, int32_t precision, void* d_phi,
                                              void* d_psi, void* stream) {
  clear_error();
  TraceRange trace("vsie_gradient_channels");
  if (!h || !d_lam || !d_phi || !d_psi || (precision != 32 && precision != 64)) {
    set_error("vsie_gradient_channels: null argument or precision not 32 / 64");
    return VSIE_ERR_ARG;
  }
  return gradient_channels(h, (const double2*)d_lam, precision, (double2*)d_phi, (double2*)d_psi,
                           (cudaStream_t)stream);
}

extern "C" vsie_status vsie_source_points(const vsie_handle* h, double* h_xyz, int32_t* h_owner,
                                          int32_t* h_class) {
  clear_error();
  TraceRange trace("vsie_source_points");
  if (!h) {
    set_error("vsie_source_points: null handle");
    return VSIE_ERR_ARG;
  }
  const Sources* cls[3] = {&h->G, &h->K, &h->F};
  int64_t off = 0;
  for (int c = 0; c < 3; ++c) {
    const Sources& S = *cls[c];
    if (!S.n) continue;
    if (h_xyz) {
      std::vector<double4_32a> ps((size_t)S.n);
      VSIE_CUDA(cudaMemcpy(ps.data(), S.pos_s, sizeof(double4_32a) * S.n, cudaMemcpyDeviceToHost));
      for (int64_t j = 0; j < S.n; ++j) {
        h_xyz[3 * (off + j)] = ps[j].x;
        h_xyz[3 * (off + j) + 1] = ps[j].y;
        h_xyz[3 * (off + j) + 2] = ps[j].z;
      }
    }
    if (h_owner) VSIE_CUDA(cudaMemcpy(h_owner + off, S.owner, sizeof(int32_t) * S.n, cudaMemcpyDeviceToHost));
    if (h_class)
      for (int64_t j = 0; j < S.n; ++j) h_class[off + j] = c;
    off += S.n;
  }
  return VSIE_OK;
}

namespace vsie {

// deterministic pseudo-random complex values in [-1, 1) (a 64-bit integer hash of i + seed)
__global__ void random_fill_kernel(double2* __restrict__ v, int64_t m, uint64_t seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + seed;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const double a = (double)(z >> 32) * (1.0 / 2147483648.0) - 1.0;
  const double b = (double)(z & 0xFFFFFFFFull) * (1.0 / 2147483648.0) - 1.0;
  v[i] = make_double2(a, b);
}

}  // namespace vsie

extern "C" vsie_status vsie_autotune(vsie_handle* h, int32_t flags, vsie_tuning* report, void* stream) {
  clear_error();
  TraceRange trace("vsie_autotune");
  if (!h || (flags & ~3) || !flags) {
    set_error("vsie_autotune: null handle or flags outside {1, 2, 3}");
    return VSIE_ERR_ARG;
  }
  vsie_tuning rep{};
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = h->n;
  const size_t cols = (flags & 2) ? 64 : 1;
  double2 *x = nullptr, *y = nullptr;
  cudaError_t e = cudaMalloc(&x, sizeof(double2) * std::max<size_t>(1, n * cols));
  if (e == cudaSuccess) e = cudaMalloc(&y, sizeof(double2) * std::max<size_t>(1, n * cols));
  if (e != cudaSuccess) {
    cudaFree(x);
    return cuda_fail(e, "cudaMalloc(autotune buffers)", __FILE__, __LINE__);
  }
  auto run = [&]() -> vsie_status {
    if (n == 0) return VSIE_OK;
    random_fill_kernel<<<(unsigned)((n * cols + 255) / 256), 256, 0, st>>>(x, (int64_t)(n * cols), 12345);
    VSIE_CUDA(cudaGetLastError());
    if (flags & 1) {
      int cand[3][2];
      double ms[3][2];
      VSIE_TRY(far_autotune(h, x, y, st, cand, ms, &rep.candidates));
      for (int c = 0; c < 3; ++c) {
        rep.far_chunk[c] = cand[c][0];
        rep.far_blocks_per_sm[c] = cand[c][1];
        rep.far_ms[c] = ms[c][0];
        rep.far_default_ms[c] = ms[c][1];
      }
      int gk_bps[2];
      double gk_ms[2];
      VSIE_TRY(far_autotune_gk(h, x, y, st, gk_bps, gk_ms, &rep.candidates));
      rep.gk_blocks_per_sm[0] = gk_bps[0];
      rep.gk_blocks_per_sm[1] = gk_bps[1];
      rep.gk_ms = gk_ms[0];
      rep.gk_sequential_ms = gk_ms[1];
    }
    if (flags & 2) {
      double ms[2];
      VSIE_TRY(batch_autotune(h, x, y, st, &rep.batch_chunk_tiles, ms, &rep.candidates));
      rep.batch_ms = ms[0];
      rep.batch_default_ms = ms[1];
    }
    VSIE_CUDA(cudaStreamSynchronize(st));
    return VSIE_OK;
  };
  const vsie_status s = run();
  cudaFree(x);
  cudaFree(y);
  if (report) *report = rep;
  return s;
}

extern "C" vsie_status vsie_set_tuning(vsie_handle* h, const vsie_tuning* t) {
  clear_error();
  TraceRange trace("vsie_set_tuning");
  if (!h || !t) {
    set_error("vsie_set_tuning: null handle or tuning");
    return VSIE_ERR_ARG;
  }
  for (int c = 0; c < 3; ++c)
    if (t->far_chunk[c] < 0 || t->far_chunk[c] > (1 << 20) || t->far_chunk[c] % 128 != 0 ||
        t->far_blocks_per_sm[c] < 0 || t->far_blocks_per_sm[c] > 64) {
      set_error("vsie_set_tuning: far_chunk must be 0 or a multiple of 128 up to 2^20 and "
                "far_blocks_per_sm in [0, 64]");
      return VSIE_ERR_ARG;
    }
  if (t->batch_chunk_tiles < 0 || t->batch_chunk_tiles > 65536 || t->gk_blocks_per_sm[0] < 0 ||
      t->gk_blocks_per_sm[1] < 0 || t->gk_blocks_per_sm[0] > 64 || t->gk_blocks_per_sm[1] > 64 ||
      (t->gk_blocks_per_sm[0] > 0) != (t->gk_blocks_per_sm[1] > 0)) {
    set_error("vsie_set_tuning: batch_chunk_tiles must be in [0, 65536] and gk_blocks_per_sm both 0 or "
              "both in [1, 64]");
    return VSIE_ERR_ARG;
  }
  for (int c = 0; c < 3; ++c) {
    h->tune.chunk[c] = t->far_chunk[c];
    h->tune.bps[c] = t->far_blocks_per_sm[c];
  }
  h->tune.bt_chunk_tiles = t->batch_chunk_tiles;
  return far_set_gk(h, t->gk_blocks_per_sm[0], t->gk_blocks_per_sm[1]);
}

extern "C" vsie_status vsie_get_tuning(const vsie_handle* h, vsie_tuning* t) {
  clear_error();
  if (!h || !t) {
    set_error("vsie_get_tuning: null handle or tuning");
    return VSIE_ERR_ARG;
  }
  vsie_tuning r{};
  for (int c = 0; c < 3; ++c) {
    r.far_chunk[c] = h->tune.chunk[c];
    r.far_blocks_per_sm[c] = h->tune.bps[c];
  }
  r.batch_chunk_tiles = h->tune.bt_chunk_tiles;
  r.gk_blocks_per_sm[0] = h->tune.gk_bps[0];
  r.gk_blocks_per_sm[1] = h->tune.gk_bps[1];
  *t = r;
  return VSIE_OK;
}

extern "C" vsie_status vsie_apply_batched_multi(vsie_handle* const* hs, int32_t nop, const void* const* d_x,
                                                void* const* d_y, int32_t nrhs, void* stream) {
  clear_error();
  TraceRange trace("vsie_apply_batched_multi");
  VSIE_TRY(check_multi_args(hs, nop, d_x, d_y, nrhs, "vsie_apply_batched_multi"));
  cudaStream_t st = (cudaStream_t)stream;
  VSIE_TRY(apply_batched_multi_launch(hs, nop, reinterpret_cast<const double2* const*>(d_x),
                                      reinterpret_cast<double2* const*>(d_y), nrhs, st));
  for (int p = 0; p < nop; ++p) VSIE_TRY(batch_status(hs[p], st));
  return VSIE_OK;
}
