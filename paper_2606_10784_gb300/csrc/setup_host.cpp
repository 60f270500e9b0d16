// Host-side setup of the AIM operators (FP64): the parts of Secs. II-III that are sparse
// bookkeeping rather than arithmetic over the grid.
//
//   * flat segments, tangents and outward normals of the closed polygon (Sec. II);
//   * Gauss-Legendre nodes per segment and the hat values at them (Eq. 7);
//   * the grid (Sec. III-A): half side L, spacing eps = 2L/(m-1), and for every node the
//     tensor-product Lagrange stencil of s points per axis (the interpolation Lambda);
//   * the composed projections P = Lambda W Phi, stored twice: grid-point-major (for the
//     anterpolation fused into the row DFT) and unknown-major (for the interpolation gather);
//   * near pairs for the near-field correction, found by spatial hashing;
//   * G^-1 (Gram matrix of Eq. 3): dense for small N, otherwise its band (the inverse of this
//     diagonally dominant cyclic tridiagonal matrix decays geometrically off the diagonal);
//   * the FFT twiddle table exp(-2 pi i t / P).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "aim_internal.h"

namespace aim {

void gauss_legendre01(int n, std::vector<double>* x, std::vector<double>* w) {
  // Newton iteration on P_n from the three-term recurrence (Golub & Welsch's classical
  // alternative; initial guesses cos(pi (i - 1/4) / (n + 1/2))).
  x->assign(n, 0.0);
  w->assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = 0.0;
      for (int j = 1; j <= n; ++j) {
        const double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
      }
      dp = n * (z * p0 - p1) / (z * z - 1.0);
      const double dz = p0 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        // one more evaluation of the derivative at the converged root
        p0 = 1.0; p1 = 0.0;
        for (int j = 1; j <= n; ++j) {
          const double p2 = p1;
          p1 = p0;
          p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
        }
        dp = n * (z * p0 - p1) / (z * z - 1.0);
        break;
      }
    }
    const double wt = 2.0 / ((1.0 - z * z) * dp * dp);
    // map [-1,1] -> [0,1]; roots come in +- pairs, z > 0 here
    (*x)[i] = 0.5 * (1.0 - z);
    (*x)[n - 1 - i] = 0.5 * (1.0 + z);
    (*w)[i] = 0.5 * wt;
    (*w)[n - 1 - i] = 0.5 * wt;
  }
}

double host_grid_half_side(const double* xy, int n, int m, int s) {
  double R = 0.0;
  for (int i = 0; i < 2 * n; ++i) R = std::max(R, std::fabs(xy[i]));
  return R / (1.0 - (s + 2.0) / (m - 1.0));
}

// Lagrange weights of s points per axis at fractional grid coordinate xi.
static inline int lagrange(double xi, int s, double* w) {
  const int base = (s % 2 == 0) ? (int)std::floor(xi) - s / 2 + 1 : (int)std::floor(xi + 0.5) - (s - 1) / 2;
  const double t = xi - base;
  for (int a = 0; a < s; ++a) {
    double num = 1.0, den = 1.0;
    for (int b = 0; b < s; ++b) {
      if (b == a) continue;
      num *= (t - b);
      den *= (double)(a - b);
    }
    w[a] = num / den;
  }
  return base;
}

static double pt_seg_dist(double px, double py, double ax, double ay, double bx, double by) {
  const double ex = bx - ax, ey = by - ay;
  double t = ((px - ax) * ex + (py - ay) * ey) / (ex * ex + ey * ey);
  t = std::min(1.0, std::max(0.0, t));
  return std::hypot(px - (ax + t * ex), py - (ay + t * ey));
}

static double seg_seg_dist(const double* p0, const double* p1, const double* q0, const double* q1) {
  return std::min(std::min(pt_seg_dist(p0[0], p0[1], q0[0], q0[1], q1[0], q1[1]),
                           pt_seg_dist(p1[0], p1[1], q0[0], q0[1], q1[0], q1[1])),
                  std::min(pt_seg_dist(q0[0], q0[1], p0[0], p0[1], p1[0], p1[1]),
                           pt_seg_dist(q1[0], q1[1], p0[0], p0[1], p1[0], p1[1])));
}

namespace {
struct Entry {
  int g;        // linear grid index iy*m + ix
  double w[kMaxProj];
};

// Accumulates the stencils of a set of points into a dense local box, then emits the
// nonzero box entries in grid order (iy major, ix minor).
struct BoxAccumulator {
  int s, m;
  int x0 = 0, y0 = 0, nx = 0, ny = 0;
  std::vector<double> box;   // ny * nx * kMaxProj
  std::vector<char> hit;
  void begin(int bx0, int by0, int bx1, int by1) {
    x0 = bx0; y0 = by0; nx = bx1 - bx0 + 1; ny = by1 - by0 + 1;
    box.assign((size_t)nx * ny * kMaxProj, 0.0);
    hit.assign((size_t)nx * ny, 0);
  }
  void add(int bx, int by, const double* wx, const double* wy, const double* val, int nval) {
    for (int b = 0; b < s; ++b)
      for (int a = 0; a < s; ++a) {
        const size_t cell = (size_t)(by + b - y0) * nx + (bx + a - x0);
        hit[cell] = 1;
        const double ww = wy[b] * wx[a];
        for (int q = 0; q < nval; ++q) box[cell * kMaxProj + q] += ww * val[q];
      }
  }
  void emit(std::vector<Entry>* out) {
    for (int yy = 0; yy < ny; ++yy)
      for (int xx = 0; xx < nx; ++xx) {
        const size_t cell = (size_t)yy * nx + xx;
        if (!hit[cell]) continue;
        Entry e;
        e.g = (y0 + yy) * m + (x0 + xx);
        for (int q = 0; q < kMaxProj; ++q) e.w[q] = box[cell * kMaxProj + q];
        out->push_back(e);
      }
  }
};
}  // namespace

aim_status host_setup(aim_ctx* ctx, HostSetup* hs) {
  const int n = ctx->n, m = ctx->m, s = ctx->s, p = ctx->p;
  const double* xy = ctx->xy.data();
  const double L = ctx->L, eps = ctx->eps;
  const bool te = ctx->form == AIM_TE_P1_GALERKIN;

  // ---- segments
  hs->dx.resize(n); hs->dy.resize(n); hs->h.resize(n);
  hs->tx.resize(n); hs->ty.resize(n); hs->nx.resize(n); hs->ny.resize(n);
  double hmax = 0.0;
  for (int e = 0; e < n; ++e) {
    const int f = (e + 1) % n;
    hs->dx[e] = xy[2 * f] - xy[2 * e];
    hs->dy[e] = xy[2 * f + 1] - xy[2 * e + 1];
    hs->h[e] = std::hypot(hs->dx[e], hs->dy[e]);
    if (!(hs->h[e] > 0.0)) return fail(AIM_EINVAL, "degenerate (zero-length) segment");
    hs->tx[e] = hs->dx[e] / hs->h[e];
    hs->ty[e] = hs->dy[e] / hs->h[e];
    hs->nx[e] = hs->ty[e];
    hs->ny[e] = -hs->tx[e];
    hmax = std::max(hmax, hs->h[e]);
  }
  gauss_legendre01(p, &hs->gx, &hs->gw);

  // ---- twiddles
  const int P = ctx->P;
  hs->tw.resize(2 * (size_t)P);
  for (int t = 0; t < P; ++t) {
    const double ang = 2.0 * M_PI * (double)t / (double)P;
    hs->tw[2 * t] = std::cos(ang);
    hs->tw[2 * t + 1] = -std::sin(ang);
  }

  // ---- projections: per unknown, the accumulated stencils of its quadrature nodes
  std::vector<double> wx(s), wy(s);
  auto stencil_of = [&](double x, double y, int* bx, int* by) {
    *bx = lagrange((x + L) / eps, s, wx.data());
    *by = lagrange((y + L) / eps, s, wy.data());
    return (*bx >= 0 && *by >= 0 && *bx + s - 1 <= m - 1 && *by + s - 1 <= m - 1);
  };

  // unknown-major lists: source side (scatter) and test side (gather)
  std::vector<std::vector<Entry>> src(n), tst;
  BoxAccumulator box{s, m};
  if (te) {
    hs->nproj = 4;
    for (int i = 0; i < n; ++i) {
      // hat i: segment i (falling piece, phi = 1 - xi) and segment i-1 (rising piece, phi = xi)
      const int segs[2] = {i, (i + n - 1) % n};
      int bxs[2][16], bys[2][16];
      int x0 = 1 << 30, y0 = 1 << 30, x1 = -1, y1 = -1;
      for (int pc = 0; pc < 2; ++pc) {
        const int e = segs[pc];
        for (int u = 0; u < p; ++u) {
          const double x = xy[2 * e] + hs->gx[u] * hs->dx[e];
          const double y = xy[2 * e + 1] + hs->gx[u] * hs->dy[e];
          if (!stencil_of(x, y, &bxs[pc][u], &bys[pc][u]))
            return fail(AIM_EINVAL, "contour too close to the grid edge for this stencil (increase L)");
          x0 = std::min(x0, bxs[pc][u]); y0 = std::min(y0, bys[pc][u]);
          x1 = std::max(x1, bxs[pc][u] + s - 1); y1 = std::max(y1, bys[pc][u] + s - 1);
        }
      }
      box.begin(x0, y0, x1, y1);
      for (int pc = 0; pc < 2; ++pc) {
        const int e = segs[pc];
        for (int u = 0; u < p; ++u) {
          const double x = xy[2 * e] + hs->gx[u] * hs->dx[e];
          const double y = xy[2 * e + 1] + hs->gx[u] * hs->dy[e];
          int bx, by;
          stencil_of(x, y, &bx, &by);
          const double wq = hs->gw[u] * hs->h[e];
          const double phi = pc == 0 ? 1.0 - hs->gx[u] : hs->gx[u];
          const double dphi = (pc == 0 ? -1.0 : 1.0) / hs->h[e];
          const double val[4] = {wq * phi, wq * dphi, wq * phi * hs->nx[e], wq * phi * hs->ny[e]};
          box.add(bx, by, wx.data(), wy.data(), val, 4);
        }
      }
      box.emit(&src[i]);
    }
  } else {
    hs->nproj = 1;
    tst.resize(n);
    for (int j = 0; j < n; ++j) {
      int x0 = 1 << 30, y0 = 1 << 30, x1 = -1, y1 = -1;
      int bxs[16], bys[16];
      for (int u = 0; u < p; ++u) {
        const double x = xy[2 * j] + hs->gx[u] * hs->dx[j];
        const double y = xy[2 * j + 1] + hs->gx[u] * hs->dy[j];
        if (!stencil_of(x, y, &bxs[u], &bys[u]))
          return fail(AIM_EINVAL, "contour too close to the grid edge for this stencil (increase L)");
        x0 = std::min(x0, bxs[u]); y0 = std::min(y0, bys[u]);
        x1 = std::max(x1, bxs[u] + s - 1); y1 = std::max(y1, bys[u] + s - 1);
      }
      box.begin(x0, y0, x1, y1);
      for (int u = 0; u < p; ++u) {
        const double x = xy[2 * j] + hs->gx[u] * hs->dx[j];
        const double y = xy[2 * j + 1] + hs->gx[u] * hs->dy[j];
        int bx, by;
        stencil_of(x, y, &bx, &by);
        const double val[1] = {hs->gw[u] * hs->h[j]};
        box.add(bx, by, wx.data(), wy.data(), val, 1);
      }
      box.emit(&src[j]);
      // collocation at the midpoint
      const double mxp = xy[2 * j] + 0.5 * hs->dx[j], myp = xy[2 * j + 1] + 0.5 * hs->dy[j];
      int bx, by;
      if (!stencil_of(mxp, myp, &bx, &by)) return fail(AIM_EINVAL, "contour too close to the grid edge");
      box.begin(bx, by, bx + s - 1, by + s - 1);
      const double one[1] = {1.0};
      box.add(bx, by, wx.data(), wy.data(), one, 1);
      box.emit(&tst[j]);
    }
  }
  const std::vector<std::vector<Entry>>& gat = te ? src : tst;

  // ---- active grid points: union of both sides, ordered by grid index
  std::vector<int> act_of((size_t)m * m, -1);
  const std::vector<std::vector<Entry>>* sides[2] = {&src, &gat};
  for (const auto* side : sides)
    for (const auto& lst : *side)
      for (const auto& e : lst) act_of[e.g] = 0;
  int n_act = 0;
  hs->row_ptr.assign(m + 1, 0);
  hs->act_ix.clear();
  hs->act_iy.clear();
  for (int g = 0; g < m * m; ++g) {
    if (act_of[g] < 0) continue;
    act_of[g] = n_act++;
    hs->act_ix.push_back(g % m);
    hs->act_iy.push_back(g / m);
    hs->row_ptr[g / m + 1]++;
  }
  for (int iy = 0; iy < m; ++iy) hs->row_ptr[iy + 1] += hs->row_ptr[iy];
  hs->n_act = n_act;
  hs->row_lo = hs->act_iy.front();
  hs->row_hi = hs->act_iy.back();

  // ---- gather CSR (unknown-major)
  hs->ga_ptr.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) hs->ga_ptr[i + 1] = hs->ga_ptr[i] + (int)gat[i].size();
  const int nga = hs->ga_ptr[n];
  hs->ga_act.resize(nga);
  for (int q = 0; q < hs->nproj; ++q) hs->ga_w[q].resize(nga);
  for (int i = 0; i < n; ++i) {
    int o = hs->ga_ptr[i];
    for (const auto& e : gat[i]) {
      hs->ga_act[o] = act_of[e.g];
      for (int q = 0; q < hs->nproj; ++q) hs->ga_w[q][o] = e.w[q];
      ++o;
    }
  }
  // ---- scatter CSR (active-point-major), by counting sort of the source entries
  hs->sc_ptr.assign(n_act + 1, 0);
  for (int j = 0; j < n; ++j)
    for (const auto& e : src[j]) hs->sc_ptr[act_of[e.g] + 1]++;
  for (int a = 0; a < n_act; ++a) hs->sc_ptr[a + 1] += hs->sc_ptr[a];
  const int nsc = hs->sc_ptr[n_act];
  hs->sc_col.resize(nsc);
  for (int q = 0; q < hs->nproj; ++q) hs->sc_w[q].resize(nsc);
  {
    std::vector<int> fill(hs->sc_ptr.begin(), hs->sc_ptr.end() - 1);
    for (int j = 0; j < n; ++j)
      for (const auto& e : src[j]) {
        const int o = fill[act_of[e.g]]++;
        hs->sc_col[o] = j;
        for (int q = 0; q < hs->nproj; ++q) hs->sc_w[q][o] = e.w[q];
      }
  }
  // source-major list for the TM near field (the TE source list equals the gather list)
  if (!te) {
    hs->sr_ptr.assign(n + 1, 0);
    for (int j = 0; j < n; ++j) hs->sr_ptr[j + 1] = hs->sr_ptr[j] + (int)src[j].size();
    hs->sr_act.resize(hs->sr_ptr[n]);
    hs->sr_w.resize(hs->sr_ptr[n]);
    for (int j = 0; j < n; ++j) {
      int o = hs->sr_ptr[j];
      for (const auto& e : src[j]) {
        hs->sr_act[o] = act_of[e.g];
        hs->sr_w[o] = e.w[0];
        ++o;
      }
    }
  }

  // ---- near pairs by spatial hashing of segment midpoints
  const double rad = ctx->near_radius;
  const double cell = rad + hmax;
  double bxmin = 1e300, bymin = 1e300, bxmax = -1e300, bymax = -1e300;
  std::vector<double> mx(n), my(n);
  for (int e = 0; e < n; ++e) {
    mx[e] = xy[2 * e] + 0.5 * hs->dx[e];
    my[e] = xy[2 * e + 1] + 0.5 * hs->dy[e];
    bxmin = std::min(bxmin, mx[e]); bxmax = std::max(bxmax, mx[e]);
    bymin = std::min(bymin, my[e]); bymax = std::max(bymax, my[e]);
  }
  const int ncx = std::max(1, (int)std::floor((bxmax - bxmin) / cell) + 1);
  const int ncy = std::max(1, (int)std::floor((bymax - bymin) / cell) + 1);
  if ((double)ncx * ncy > 4.0e7) return fail(AIM_EINVAL, "near radius too small relative to the contour size");
  std::vector<int> cstart((size_t)ncx * ncy + 1, 0), cseg(n), ccell(n);
  for (int e = 0; e < n; ++e) {
    const int cx = std::min(ncx - 1, (int)std::floor((mx[e] - bxmin) / cell));
    const int cy = std::min(ncy - 1, (int)std::floor((my[e] - bymin) / cell));
    ccell[e] = cy * ncx + cx;
    cstart[ccell[e] + 1]++;
  }
  for (size_t c = 0; c < (size_t)ncx * ncy; ++c) cstart[c + 1] += cstart[c];
  {
    std::vector<int> fill(cstart.begin(), cstart.end() - 1);
    for (int e = 0; e < n; ++e) cseg[fill[ccell[e]]++] = e;
  }
  auto for_candidates = [&](double px, double py, auto&& fn) {
    const int cx = std::min(ncx - 1, std::max(0, (int)std::floor((px - bxmin) / cell)));
    const int cy = std::min(ncy - 1, std::max(0, (int)std::floor((py - bymin) / cell)));
    for (int yy = std::max(0, cy - 1); yy <= std::min(ncy - 1, cy + 1); ++yy)
      for (int xx = std::max(0, cx - 1); xx <= std::min(ncx - 1, cx + 1); ++xx) {
        const int c = yy * ncx + xx;
        for (int q = cstart[c]; q < cstart[c + 1]; ++q) fn(cseg[q]);
      }
  };

  std::vector<std::vector<int>> rows(n);
  if (te) {
    for (int e = 0; e < n; ++e) {
      const double* p0 = &xy[2 * e];
      const double* p1 = &xy[2 * ((e + 1) % n)];
      for_candidates(mx[e], my[e], [&](int f) {
        const double* q0 = &xy[2 * f];
        const double* q1 = &xy[2 * ((f + 1) % n)];
        if (seg_seg_dist(p0, p1, q0, q1) <= rad) {
          const int hi[2] = {e, (e + 1) % n}, hj[2] = {f, (f + 1) % n};
          for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) rows[hi[a]].push_back(hj[b]);
        }
      });
    }
  } else {
    for (int i = 0; i < n; ++i) {
      for_candidates(mx[i], my[i], [&](int j) {
        const double* q0 = &xy[2 * j];
        const double* q1 = &xy[2 * ((j + 1) % n)];
        if (pt_seg_dist(mx[i], my[i], q0[0], q0[1], q1[0], q1[1]) <= rad) rows[i].push_back(j);
      });
    }
  }
  hs->near_ptr.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    auto& r = rows[i];
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
    hs->near_ptr[i + 1] = hs->near_ptr[i] + (int)r.size();
  }
  hs->near_col.resize(hs->near_ptr[n]);
  for (int i = 0; i < n; ++i) std::copy(rows[i].begin(), rows[i].end(), hs->near_col.begin() + hs->near_ptr[i]);

  // segment pairs needed by the exact near entries
  hs->seg_e.clear(); hs->seg_f.clear(); hs->pair_seg_idx.clear();
  if (te) {
    std::unordered_map<long long, int> idx;
    idx.reserve((size_t)hs->near_ptr[n] * 2);
    hs->pair_seg_idx.resize((size_t)hs->near_ptr[n] * 4);
    for (int i = 0; i < n; ++i)
      for (int q = hs->near_ptr[i]; q < hs->near_ptr[i + 1]; ++q) {
        const int j = hs->near_col[q];
        const int es[4] = {i, i, (i + n - 1) % n, (i + n - 1) % n};
        const int fs[4] = {j, (j + n - 1) % n, j, (j + n - 1) % n};
        for (int c = 0; c < 4; ++c) {
          const long long key = (long long)es[c] * n + fs[c];
          auto it = idx.find(key);
          int id;
          if (it == idx.end()) {
            id = (int)hs->seg_e.size();
            idx.emplace(key, id);
            hs->seg_e.push_back(es[c]);
            hs->seg_f.push_back(fs[c]);
          } else {
            id = it->second;
          }
          hs->pair_seg_idx[(size_t)q * 4 + c] = id;
        }
      }
  }

  // ---- G^-1 (TE)
  if (te) {
    // cyclic tridiagonal: diag_i = (h_{i-1}+h_i)/3, G[i][i+1] = G[i+1][i] = h_i/6
    auto diag = [&](int i) { return (hs->h[(i + n - 1) % n] + hs->h[i]) / 3.0; };
    auto off = [&](int i) { return hs->h[i] / 6.0; };   // couples i and i+1
    if (n <= kGramDenseMax) {
      // dense inverse: Sherman-Morrison on the cyclic system, one Thomas solve per column
      const int blo = n / 2;
      hs->gram_band = blo;
      hs->gram_inv.assign((size_t)n * n, 0.0);
      std::vector<double> a(n), b(n), c(n);
      for (int i = 0; i < n; ++i) {
        b[i] = diag(i);
        a[i] = off((i + n - 1) % n);   // G[i][i-1]
        c[i] = off(i);                 // G[i][i+1]
      }
      const double alpha = c[n - 1], beta = a[0];   // G[n-1][0], G[0][n-1]
      const double gamma = -b[0];
      std::vector<double> bb(b);
      bb[0] = b[0] - gamma;
      bb[n - 1] = b[n - 1] - alpha * beta / gamma;
      auto thomas = [&](const std::vector<double>& rhs, std::vector<double>* x) {
        std::vector<double> cp(n), dp(n);
        cp[0] = c[0] / bb[0];
        dp[0] = rhs[0] / bb[0];
        for (int i = 1; i < n; ++i) {
          const double den = bb[i] - a[i] * cp[i - 1];
          cp[i] = c[i] / den;
          dp[i] = (rhs[i] - a[i] * dp[i - 1]) / den;
        }
        (*x)[n - 1] = dp[n - 1];
        for (int i = n - 2; i >= 0; --i) (*x)[i] = dp[i] - cp[i] * (*x)[i + 1];
      };
      std::vector<double> u(n, 0.0), z(n), y(n), rhs(n);
      u[0] = gamma;
      u[n - 1] = alpha;
      thomas(u, &z);
      const double vz = z[0] + beta / gamma * z[n - 1];
      for (int col = 0; col < n; ++col) {
        std::fill(rhs.begin(), rhs.end(), 0.0);
        rhs[col] = 1.0;
        thomas(rhs, &y);
        const double vy = y[0] + beta / gamma * y[n - 1];
        const double f = vy / (1.0 + vz);
        // column col of G^-1 = row col (symmetric); store row col at offsets d = 0..n-1 from col-blo
        for (int d = 0; d < n; ++d) {
          int j = col - blo + d;
          j = ((j % n) + n) % n;
          hs->gram_inv[(size_t)col * n + d] = y[j] - f * z[j];
        }
      }
    } else {
      const int B = kGramBand, Wd = 64, len = 2 * Wd + 1;
      hs->gram_band = B;
      hs->gram_inv.assign((size_t)n * (2 * B + 1), 0.0);
      std::vector<double> a(len), b(len), c(len), cp(len), dp(len), x(len);
      for (int i = 0; i < n; ++i) {
        for (int t = 0; t < len; ++t) {
          const int g = ((i - Wd + t) % n + n) % n;
          b[t] = diag(g);
          a[t] = off((g + n - 1) % n);
          c[t] = off(g);
        }
        // solve the window system with e_center (boundary couplings dropped)
        cp[0] = c[0] / b[0];
        dp[0] = (Wd == 0) ? 1.0 / b[0] : 0.0;
        for (int t = 1; t < len; ++t) {
          const double den = b[t] - a[t] * cp[t - 1];
          cp[t] = c[t] / den;
          dp[t] = ((t == Wd ? 1.0 : 0.0) - a[t] * dp[t - 1]) / den;
        }
        x[len - 1] = dp[len - 1];
        for (int t = len - 2; t >= 0; --t) x[t] = dp[t] - cp[t] * x[t + 1];
        for (int d = 0; d < 2 * B + 1; ++d) hs->gram_inv[(size_t)i * (2 * B + 1) + d] = x[Wd - B + d];
      }
    }
  }
  return AIM_OK;
}

}  // namespace aim
