// Host code: the pre-tabulated grid pair force F^P of Sec. II.B.1 (Eq. LC)
// and the ES kernel normalisation of App. B (Eq. eskernel).
//
// f^P(r) is the component along (x_i - x_j)/r of the force the grid pipeline
// (spread j, unbounded-domain Poisson, -grad on faces, interpolate at i)
// exerts on unit charge i from unit charge j with l_B = 1, averaged over a
// fixed sample set: 8 sub-cell offsets of x_j, ((a + 1/2)/2 per axis, a in
// {0, 1}), times 13 directions (the cube's axes, face diagonals and body
// diagonals, one of each +/- pair).  The unbounded-domain solve uses the
// lattice Green's function of the 7-point Laplacian,
//     G(n) = int_0^inf prod_d e^{-2t} I_{n_d}(2t) dt,
// with e^{-x} I_n(x) from its power series (all terms positive) for
// x <= 600 and from the Hankel asymptotic series beyond, integrated by
// composite Gauss-Legendre on [0, T] and in u = t^{-1/2} on the tail.
#include <cmath>
#include <map>
#include <string>
#include <tuple>
#include <vector>
#include <algorithm>
#include "internal.h"

namespace discos {

namespace {

// e^{-x} I_n(x), n >= 0, x >= 0
double ive(int n, double x) {
  if (x == 0.0) return n == 0 ? 1.0 : 0.0;
  if (x <= 600.0) {
    double lt = -x + n * std::log(0.5 * x) - std::lgamma(n + 1.0);
    double term = std::exp(lt);
    double sum = term;
    double q = 0.25 * x * x;
    for (int k = 0; k < 100000; ++k) {
      term *= q / ((k + 1.0) * (k + 1.0 + n));
      sum += term;
      if (k > 0.5 * x && term < 1e-18 * sum) break;
    }
    return sum;
  }
  // Hankel expansion: (2 pi x)^-1/2 sum_k (-1)^k a_k(n) / x^k,
  // a_k = prod_{j=1..k} (4n^2 - (2j-1)^2) / (k! 8^k)
  double mu = 4.0 * n * n;
  double term = 1.0, sum = 1.0, prev = 1e300;
  for (int k = 1; k < 60; ++k) {
    term *= -(mu - (2.0 * k - 1.0) * (2.0 * k - 1.0)) / (k * 8.0 * x);
    if (std::fabs(term) > prev) break;
    sum += term;
    prev = std::fabs(term);
    if (prev < 1e-18) break;
  }
  return sum / std::sqrt(2.0 * M_PI * x);
}

// 20-point Gauss-Legendre nodes/weights on [-1, 1], computed by Newton's
// iteration on the Legendre recurrence.
struct GL {
  double x[20], w[20];
  GL() {
    const int n = 20;
    for (int i = 0; i < n; ++i) {
      double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        double dp = n * (z * p1 - p0) / (z * z - 1.0);
        double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
};

double lattice_green(int a, int b, int c) {
  static const GL gl;
  a = std::abs(a); b = std::abs(b); c = std::abs(c);
  auto f = [&](double t) { return ive(a, 2 * t) * ive(b, 2 * t) * ive(c, 2 * t); };
  const double T = 30.0;
  const int panels = 120;
  double head = 0.0;
  for (int p = 0; p < panels; ++p) {
    // denser panels near t = 0 where the integrand varies fastest
    double t0 = T * std::pow((double)p / panels, 2.0), t1 = T * std::pow((double)(p + 1) / panels, 2.0);
    double hm = 0.5 * (t1 - t0), cm = 0.5 * (t1 + t0);
    for (int i = 0; i < 20; ++i) head += gl.w[i] * hm * f(cm + hm * gl.x[i]);
  }
  // tail: t = 1/u^2, dt = -2 du / u^3, u in (0, 1/sqrt(T)]
  double tail = 0.0;
  const double U = 1.0 / std::sqrt(T);
  const int tp = 8;
  for (int p = 0; p < tp; ++p) {
    double u0 = U * p / tp, u1 = U * (p + 1) / tp;
    double hm = 0.5 * (u1 - u0), cm = 0.5 * (u1 + u0);
    for (int i = 0; i < 20; ++i) {
      double u = cm + hm * gl.x[i];
      tail += gl.w[i] * hm * f(1.0 / (u * u)) * 2.0 / (u * u * u);
    }
  }
  return head + tail;
}

}  // namespace

double es_normalisation(int w, double beta) {
  // int_{-a}^{a} exp(beta (sqrt(1 - (z/a)^2) - 1)) dz with z = a sin(theta)
  static const GL gl;
  double a = 0.5 * w;
  double sum = 0.0;
  const int panels = 64;
  for (int p = 0; p < panels; ++p) {
    double t0 = -0.5 * M_PI + M_PI * p / panels, t1 = -0.5 * M_PI + M_PI * (p + 1) / panels;
    double hm = 0.5 * (t1 - t0), cm = 0.5 * (t1 + t0);
    for (int i = 0; i < 20; ++i) {
      double th = cm + hm * gl.x[i];
      sum += gl.w[i] * hm * std::exp(beta * (std::cos(th) - 1.0)) * a * std::cos(th);
    }
  }
  return sum;
}

bool build_fp_table(const KernelParams& kp, double psi, int n_tab, double* out, std::string* err) {
  const int w = kp.w;
  const int R = w + 3 + (int)std::ceil(psi);
  const int S = 2 * R + 1;
  std::vector<double> G((size_t)S * S * S);
  std::map<std::tuple<int, int, int>, double> cache;
  for (int c = -R; c <= R; ++c)
    for (int b = -R; b <= R; ++b)
      for (int a = -R; a <= R; ++a) {
        int v[3] = {std::abs(a), std::abs(b), std::abs(c)};
        std::sort(v, v + 3);
        auto key = std::make_tuple(v[0], v[1], v[2]);
        auto it = cache.find(key);
        double g;
        if (it == cache.end()) {
          g = lattice_green(v[0], v[1], v[2]);
          cache[key] = g;
        } else {
          g = it->second;
        }
        G[((size_t)(c + R) * S + (b + R)) * S + (a + R)] = g;
      }
  static const double dirs[13][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, -1, 0}, {1, 0, 1}, {1, 0, -1},
                                     {0, 1, 1}, {0, 1, -1}, {1, 1, 1}, {1, 1, -1}, {1, -1, 1}, {-1, 1, 1}};
  out[0] = 0.0;
  std::vector<double> phi;
  for (int k = 1; k <= n_tab; ++k) {
    double r = k * psi / n_tab;
    double acc = 0.0;
    int ns = 0;
    for (int az = 0; az < 2; ++az)
      for (int ay = 0; ay < 2; ++ay)
        for (int ax = 0; ax < 2; ++ax) {
          double xj[3] = {20.0 + (ax + 0.5) / 2, 20.0 + (ay + 0.5) / 2, 20.0 + (az + 0.5) / 2};
          for (int di = 0; di < 13; ++di) {
            double nrm = std::sqrt(dirs[di][0] * dirs[di][0] + dirs[di][1] * dirs[di][1] + dirs[di][2] * dirs[di][2]);
            double u[3] = {dirs[di][0] / nrm, dirs[di][1] / nrm, dirs[di][2] / nrm};
            double xi[3] = {xj[0] + r * u[0], xj[1] + r * u[1], xj[2] + r * u[2]};
            // source: cells p (centres p + 1/2)
            int ps[3];
            double ws[3][8];
            for (int d = 0; d < 3; ++d) {
              double s = xj[d] - 0.5;
              ps[d] = stencil_start(s, w);
              for (int l = 0; l < w; ++l) ws[d][l] = kval(s - (ps[d] + l), kp);
            }
            // target block: cells [fs - 1, fs + w - 1], fs = first face of i's face stencil
            int c0[3];
            double cw[3][9], ew[3][9];
            for (int d = 0; d < 3; ++d) {
              c0[d] = stencil_start(xi[d], w) - 1;
              for (int l = 0; l <= w; ++l) {
                int c = c0[d] + l;
                cw[d][l] = kval(xi[d] - (c + 0.5), kp);
                ew[d][l] = kval(xi[d] - (double)(c + 1), kp) - kval(xi[d] - (double)c, kp);
              }
            }
            double F[3] = {0, 0, 0};
            for (int lz = 0; lz <= w; ++lz)
              for (int ly = 0; ly <= w; ++ly)
                for (int lx = 0; lx <= w; ++lx) {
                  int cx = c0[0] + lx, cy = c0[1] + ly, cz = c0[2] + lz;
                  double ph = 0.0;
                  for (int pz = 0; pz < w; ++pz) {
                    int dz = cz - (ps[2] + pz);
                    for (int py = 0; py < w; ++py) {
                      int dy = cy - (ps[1] + py);
                      double wzy = ws[2][pz] * ws[1][py];
                      const double* row = &G[((size_t)(dz + R) * S + (dy + R)) * S + R];
                      for (int px = 0; px < w; ++px) {
                        int dx = cx - (ps[0] + px);
                        ph += row[dx] * wzy * ws[0][px];
                      }
                    }
                  }
                  ph *= 4.0 * M_PI;
                  F[0] += ph * ew[0][lx] * cw[1][ly] * cw[2][lz];
                  F[1] += ph * cw[0][lx] * ew[1][ly] * cw[2][lz];
                  F[2] += ph * cw[0][lx] * cw[1][ly] * ew[2][lz];
                }
            acc += F[0] * u[0] + F[1] * u[1] + F[2] * u[2];
            ++ns;
          }
        }
    out[k] = acc / ns;
  }
  (void)err;
  return true;
}

}  // namespace discos

extern "C" discos_status discos_fp_table(int kernel, int es_w, double es_beta, double psi, int n_tab, double* out) {
  if (!out || n_tab < 2 || !(psi > 0.0)) return DISCOS_ERR_INVALID_ARG;
  discos::KernelParams kp{};
  kp.kind = kernel;
  if (kernel == DISCOS_KERNEL_PESKIN4) kp.w = 4;
  else if (kernel == DISCOS_KERNEL_PESKIN6) kp.w = 6;
  else if (kernel == DISCOS_KERNEL_ES) {
    if (es_w < 4 || es_w > 7) return DISCOS_ERR_INVALID_ARG;
    kp.w = es_w;
    kp.alpha = 0.5 * es_w;
    kp.beta = es_beta;
    kp.inv_norm = 1.0 / discos::es_normalisation(es_w, es_beta);
  } else {
    return DISCOS_ERR_INVALID_ARG;
  }
  std::string err;
  return discos::build_fp_table(kp, psi, n_tab, out, &err) ? DISCOS_OK : DISCOS_ERR_INVALID_ARG;
}
