// 1D reference tables: Gauss-Lobatto-Legendre nodes/weights, Gauss-Legendre
// rules and Lagrange basis tables. Host code, computed once per context.
//
// The paper fixes neither basis nor quadrature (Sec. 2 only asks for degree-p
// polynomials per element and face); this library uses tensor-product
// Lagrange polynomials on GLL nodes and Gauss quadrature exact for every
// product that appears in the local equations.
#include <cmath>
#include <stdexcept>

#include "ehdg_internal.h"

namespace ehdg {

namespace {

// Legendre P_n(x) and P_{n-1}(x) by the three-term recurrence.
void legendre(int n, double x, double* pn, double* pn1) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *pn = 1.0; *pn1 = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  *pn1 = p0;
}

}  // namespace

void gauss_rule(int q, std::vector<double>* x, std::vector<double>* w) {
  x->assign(q, 0.0);
  w->assign(q, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < q; ++i) {
    // Chebyshev-like initial guess, ascending order
    double z = -std::cos(pi * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double pn, pn1;
      legendre(q, z, &pn, &pn1);
      double dp = q * (z * pn - pn1) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    double pn, pn1;
    legendre(q, z, &pn, &pn1);
    double dp = q * (z * pn - pn1) / (z * z - 1.0);
    (*x)[i] = z;
    (*w)[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

void gll_rule(int p, std::vector<double>* x, std::vector<double>* w) {
  x->assign(p + 1, 0.0);
  w->assign(p + 1, 0.0);
  const double pi = 3.14159265358979323846;
  (*x)[0] = -1.0;
  (*x)[p] = 1.0;
  // interior nodes: roots of P_p', Newton with P_p'' from Legendre's equation
  for (int j = 1; j < p; ++j) {
    double z = -std::cos(pi * j / p);
    for (int it = 0; it < 100; ++it) {
      double pn, pn1;
      legendre(p, z, &pn, &pn1);
      double d1 = p * (z * pn - pn1) / (z * z - 1.0);
      double d2 = (2.0 * z * d1 - p * (p + 1.0) * pn) / (1.0 - z * z);
      double dz = d1 / d2;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    (*x)[j] = z;
  }
  for (int j = 0; j <= p; ++j) {
    double pn, pn1;
    legendre(p, (*x)[j], &pn, &pn1);
    (*w)[j] = 2.0 / (p * (p + 1.0) * pn * pn);
  }
}

void build_ref1d(int p, int q, Ref1D* o) {
  o->p = p;
  o->q = q;
  gll_rule(p, &o->r, &o->wr);
  gauss_rule(q, &o->xi, &o->om);
  const int n1 = p + 1;
  o->L.assign(q * n1, 0.0);
  o->D.assign(q * n1, 0.0);
  o->Lend.assign(2 * n1, 0.0);
  auto lag = [&](double x, int a) {
    double v = 1.0;
    for (int b = 0; b < n1; ++b)
      if (b != a) v *= (x - o->r[b]) / (o->r[a] - o->r[b]);
    return v;
  };
  auto dlag = [&](double x, int a) {
    double s = 0.0;
    for (int m = 0; m < n1; ++m) {
      if (m == a) continue;
      double t = 1.0 / (o->r[a] - o->r[m]);
      for (int b = 0; b < n1; ++b)
        if (b != a && b != m) t *= (x - o->r[b]) / (o->r[a] - o->r[b]);
      s += t;
    }
    return s;
  };
  for (int g = 0; g < q; ++g)
    for (int a = 0; a < n1; ++a) {
      o->L[g * n1 + a] = lag(o->xi[g], a);
      o->D[g * n1 + a] = dlag(o->xi[g], a);
    }
  for (int a = 0; a < n1; ++a) {
    o->Lend[a] = lag(-1.0, a);
    o->Lend[n1 + a] = lag(1.0, a);
  }
}

}  // namespace ehdg
