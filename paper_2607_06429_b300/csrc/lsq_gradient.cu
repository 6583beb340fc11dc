// Density gradient for element-wise density (host code, create time): grad(alpha) of the
// adjoint double layer (Eq. vsie, T term) is not defined by an element-wise alpha, so the
// library offers the least-squares reading: over the face neighbours f of tetrahedron e in
// the same subdomain,
//     g_e = argmin_g sum_f (alpha_f - alpha_e - g . (c_f - c_e))^2,      c = centroids,
// the minimum-norm minimiser when the neighbours span fewer than three directions (the
// pseudo-inverse of D = [c_f - c_e], singular values below 1e-6 of the largest dropped:
// formed from D^T D, whose rounding leaves ~1e-16 of the largest eigenvalue where D is
// exactly rank deficient, so the cut sits well above that and far below any real spread),
// 0 without neighbours.  g is linear in alpha, g = W alpha; the adjoint W^T carries a
// gradient with respect to grad(alpha) back to alpha (the chain rule of a density
// gradient).

#include <algorithm>
#include <array>
#include <cmath>
#include <vector>

#include "vsie_internal.h"

namespace vsie {
namespace {

struct Stencil {
  std::vector<int64_t> first;   // n_tet + 1
  std::vector<int32_t> nb;      // neighbours
  std::vector<double> coef;     // 3 per neighbour: P[:, q] (g_e = sum_q P[:, q] (alpha_f - alpha_e))
};

// eigen-decomposition of a symmetric 3 x 3 matrix by cyclic Jacobi rotations
void jacobi3(double a[3][3], double ev[3], double V[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 50; ++sweep) {
    const double off = std::fabs(a[0][1]) + std::fabs(a[0][2]) + std::fabs(a[1][2]);
    const double dia = std::fabs(a[0][0]) + std::fabs(a[1][1]) + std::fabs(a[2][2]);
    if (off <= 1e-300 || off <= 1e-18 * dia) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (a[p][q] == 0.0) continue;
        const double th = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < 3; ++k) {  // A <- A J
          const double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {  // A <- J^T A
          const double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < 3; ++i) ev[i] = a[i][i];
}

vsie_status build_stencil(const vsie_mesh* mesh, const int8_t* dom, Stencil& S) {
  const int64_t nt = mesh->n_tet;
  const int32_t* tet = mesh->tet;
  // faces as sorted vertex triples; two tetrahedra sharing a face are adjacent
  std::vector<std::pair<std::array<int32_t, 3>, int32_t>> faces;
  faces.reserve((size_t)nt * 4);
  for (int64_t e = 0; e < nt; ++e)
    for (int f = 0; f < 4; ++f) {
      std::array<int32_t, 3> k;
      int q = 0;
      for (int j = 0; j < 4; ++j)
        if (j != f) k[q++] = tet[4 * e + j];
      std::sort(k.begin(), k.end());
      faces.push_back({k, (int32_t)e});
    }
  std::sort(faces.begin(), faces.end());
  std::vector<std::vector<int32_t>> nb((size_t)nt);
  for (size_t i = 0; i + 1 < faces.size(); ++i)
    if (faces[i].first == faces[i + 1].first) {
      const int32_t a = faces[i].second, b = faces[i + 1].second;
      if (!dom || dom[a] == dom[b]) {
        nb[a].push_back(b);
        nb[b].push_back(a);
      }
    }
  std::vector<double> cen((size_t)nt * 3, 0.0);
  for (int64_t e = 0; e < nt; ++e)
    for (int j = 0; j < 4; ++j)
      for (int d = 0; d < 3; ++d) cen[3 * e + d] += 0.25 * mesh->vert[3 * (int64_t)tet[4 * e + j] + d];
  S.first.assign((size_t)nt + 1, 0);
  for (int64_t e = 0; e < nt; ++e) {
    std::sort(nb[e].begin(), nb[e].end());
    S.first[e + 1] = S.first[e] + (int64_t)nb[e].size();
  }
  S.nb.resize((size_t)S.first[nt]);
  S.coef.assign((size_t)S.first[nt] * 3, 0.0);
  for (int64_t e = 0; e < nt; ++e) {
    const size_t k = nb[e].size();
    if (!k) continue;
    std::vector<double> Dm(k * 3);
    double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (size_t q = 0; q < k; ++q)
      for (int d = 0; d < 3; ++d) Dm[3 * q + d] = cen[3 * (size_t)nb[e][q] + d] - cen[3 * e + d];
    for (size_t q = 0; q < k; ++q)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i][j] += Dm[3 * q + i] * Dm[3 * q + j];
    // pseudo-inverse of D via M = D^T D = V diag(ev) V^T: P = V diag(1/ev) V^T D^T, with
    // the eigenvalues (squared singular values) below (1e-6)^2 of the largest dropped
    double ev[3], V[3][3];
    jacobi3(M, ev, V);
    const double emax = std::max(ev[0], std::max(ev[1], ev[2]));
    double Minv[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int m = 0; m < 3; ++m) {
      if (!(ev[m] > 1e-12 * emax) || !(emax > 0.0)) continue;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Minv[i][j] += V[i][m] * V[j][m] / ev[m];
    }
    for (size_t q = 0; q < k; ++q) {
      const int64_t o = S.first[e] + (int64_t)q;
      S.nb[o] = nb[e][q];
      for (int i = 0; i < 3; ++i)
        S.coef[3 * o + i] = Minv[i][0] * Dm[3 * q] + Minv[i][1] * Dm[3 * q + 1] + Minv[i][2] * Dm[3 * q + 2];
    }
  }
  return VSIE_OK;
}

vsie_status check_mesh(const vsie_mesh* mesh, const char* who) {
  if (!mesh || mesh->n_tet < 0 || (mesh->n_tet > 0 && (!mesh->tet || !mesh->vert))) {
    set_error(std::string(who) + ": null mesh arrays");
    return VSIE_ERR_ARG;
  }
  for (int64_t i = 0; i < 4 * mesh->n_tet; ++i)
    if (mesh->tet[i] < 0 || mesh->tet[i] >= mesh->n_vert) {
      set_error(std::string(who) + ": tetrahedron vertex index out of range");
      return VSIE_ERR_MESH;
    }
  return VSIE_OK;
}

}  // namespace
}  // namespace vsie

using namespace vsie;

extern "C" vsie_status vsie_lsq_grad_alpha(const vsie_mesh* mesh, const int8_t* tet_domain, const double* alpha,
                                           double* grad_alpha) {
  clear_error();
  TraceRange trace("vsie_lsq_grad_alpha");
  VSIE_TRY(check_mesh(mesh, "vsie_lsq_grad_alpha"));
  if (!alpha || !grad_alpha) {
    set_error("vsie_lsq_grad_alpha: null alpha or output");
    return VSIE_ERR_ARG;
  }
  Stencil S;
  VSIE_TRY(build_stencil(mesh, tet_domain, S));
  for (int64_t e = 0; e < mesh->n_tet; ++e) {
    double g[3] = {0.0, 0.0, 0.0};
    for (int64_t o = S.first[e]; o < S.first[e + 1]; ++o) {
      const double da = alpha[S.nb[o]] - alpha[e];
      for (int i = 0; i < 3; ++i) g[i] += S.coef[3 * o + i] * da;
    }
    for (int i = 0; i < 3; ++i) grad_alpha[3 * e + i] = g[i];
  }
  return VSIE_OK;
}

extern "C" vsie_status vsie_lsq_grad_alpha_adjoint(const vsie_mesh* mesh, const int8_t* tet_domain,
                                                   const double* d_grad, double* d_alpha) {
  clear_error();
  TraceRange trace("vsie_lsq_grad_alpha_adjoint");
  VSIE_TRY(check_mesh(mesh, "vsie_lsq_grad_alpha_adjoint"));
  if (!d_grad || !d_alpha) {
    set_error("vsie_lsq_grad_alpha_adjoint: null input or output");
    return VSIE_ERR_ARG;
  }
  Stencil S;
  VSIE_TRY(build_stencil(mesh, tet_domain, S));
  std::fill(d_alpha, d_alpha + mesh->n_tet, 0.0);
  for (int64_t e = 0; e < mesh->n_tet; ++e)
    for (int64_t o = S.first[e]; o < S.first[e + 1]; ++o) {
      double w = 0.0;  // (W^T)[f, e] applied: P[:, q] . d_grad_e
      for (int i = 0; i < 3; ++i) w += S.coef[3 * o + i] * d_grad[3 * e + i];
      d_alpha[S.nb[o]] += w;
      d_alpha[e] -= w;
    }
  return VSIE_OK;
}
