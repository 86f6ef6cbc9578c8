// Tile bodies of the once-per-step kernels (32 elements x kStepT row
// groups): the step's right-hand side (G = P w, then Gy = Ey G and the
// element values Y0 = Ey u^n at the sweep's rows) and the end-of-step
// reconstruction u^{k+1} = G + H uhat^k (Crank-Nicolson: 2 v - u^n). The
// single-problem kernels and the batched step run this code, so their
// results agree bit for bit.
#pragma once

#include <cuda_runtime.h>

#include "ehdg_internal.h"

namespace ehdg {

constexpr int kStepT = 4;

struct StepParams {
  int64_t nel;
  int n, NQFS, KE, shared;
  double ucoef;                 // 1/dt_eff, or 0 for steady
  int have_force, force_avg;    // force_avg: use 0.5 (f_old + f) (Crank-Nicolson)
  const double* P;
  const double* u;
  const double* force;
  const double* force_old;
  const int* ey_idx;
  const double* ey_val;
  const int* rows;              // shared operator: output rows of every element
  int n_rows;
  const uint8_t* rowid;         // per-element operator: [NQFS][nel] row of each slot
  const uint8_t* nrows;         // [nel] slots in use
  int g_ready;                  // 1: G = P w already computed (tensor-core step)
  // hexahedra whose sweep rows are whole faces (one shared transport
  // operator, q = p + 1): Y0 and Gy by two 1D passes per row face instead of
  // the dense (p+1)^2-term rows of Ey
  int sf_ey, sf_nf, sf_p1, Nqf;
  int sf_face[3];               // local face of each row face
  int sf_base[3], sf_sa[3], sf_sb[3];   // its node index: base + ia sa + ib sb
  double sfL[16];               // [g][i] Lagrange basis i at Gauss point g
  double* G;
  double* Gy;                   // [slot][nel], slot order of the element sweep
  double* Y;
  // warm start (or null): while *warm is 1 the next initial trace comes from
  // the previous step's final trace, so Y0 = Ey u^n is not formed
  const int* warm;
};

// Psh: a shared operator P [n][n]; w, g: [n][32] scratch; sfw: the face
// passes' scratch [sf_nf q][p+1][2][32] (sf_ey only).
__device__ __forceinline__ void step_tile(const StepParams& s, const double* Psh, double* w,
                                          double* g, double* sfw, int64_t tile) {
  const int lane = threadIdx.x, t = threadIdx.y;
  const int n = s.n;
  const int64_t ne = s.nel;
  const int64_t e = tile * 32 + lane;
  const bool live = e < ne;
  __syncthreads();
  if (s.g_ready) {
    // G = P w came from the FP64-accurate tensor-core product
    for (int r = t; r < n; r += kStepT) g[r * 32 + lane] = live ? s.G[r * ne + e] : 0.0;
  } else {
    for (int c = t; c < n; c += kStepT) {
      double v = 0.0;
      if (live) {
        v = s.u[c * ne + e] * s.ucoef;
        if (s.have_force)
          v += s.force_avg ? 0.5 * (s.force[c * ne + e] + s.force_old[c * ne + e])
                           : s.force[c * ne + e];
      }
      w[c * 32 + lane] = v;
    }
    __syncthreads();
    for (int r = t; r < n; r += kStepT) {
      double a0 = 0.0, a1 = 0.0;
      if (s.shared) {
        const double* Pr = Psh + r * n;
        int c = 0;
        for (; c + 1 < n; c += 2) {
          a0 = fma(Pr[c], w[c * 32 + lane], a0);
          a1 = fma(Pr[c + 1], w[(c + 1) * 32 + lane], a1);
        }
        if (c < n) a0 = fma(Pr[c], w[c * 32 + lane], a0);
      } else if (live) {
        const double* Pr = s.P + (int64_t)r * n * ne + e;
        int c = 0;
        for (; c + 1 < n; c += 2) {
          a0 = fma(Pr[c * ne], w[c * 32 + lane], a0);
          a1 = fma(Pr[(c + 1) * ne], w[(c + 1) * 32 + lane], a1);
        }
        if (c < n) a0 = fma(Pr[c * ne], w[c * 32 + lane], a0);
      }
      const double acc = a0 + a1;
      g[r * 32 + lane] = acc;
      if (live) s.G[r * ne + e] = acc;
    }
  }
  __syncthreads();
  const bool want_y0 = !(s.warm && *s.warm);
  if (s.sf_ey) {
    // Y0 = Ey u^n and Gy = Ey G on each row face: the face's nodes are a
    // (p+1) x (p+1) grid (tangential axes a < b), and Ey there is L x L, so
    // pass 1 contracts axis a for each Gauss index g0 along a, pass 2 axis b
    const int p1 = s.sf_p1, q = s.sf_p1, nit = s.sf_nf * q;
    for (int it = t; it < nit; it += kStepT) {
      const int rf = it / q, g0 = it - rf * q;
      const double* La = s.sfL + g0 * p1;
      for (int ib = 0; ib < p1; ++ib) {
        double y = 0.0, gg = 0.0;
        if (live) {
          const int i0 = s.sf_base[rf] + ib * s.sf_sb[rf];
          if (want_y0) {
            for (int ia = 0; ia < p1; ++ia) {
              const int i = i0 + ia * s.sf_sa[rf];
              y = fma(La[ia], s.u[i * ne + e], y);
              gg = fma(La[ia], g[i * 32 + lane], gg);
            }
          } else {
            for (int ia = 0; ia < p1; ++ia) gg = fma(La[ia], g[(i0 + ia * s.sf_sa[rf]) * 32 + lane], gg);
          }
        }
        sfw[((it * p1 + ib) * 2) * 32 + lane] = y;
        sfw[((it * p1 + ib) * 2 + 1) * 32 + lane] = gg;
      }
    }
    __syncthreads();
    if (!live) return;
    for (int it = t; it < nit; it += kStepT) {
      const int rf = it / q, g1 = it - rf * q;
      const double* Lb = s.sfL + g1 * p1;
      for (int g0 = 0; g0 < q; ++g0) {
        const double* src = sfw + ((rf * q + g0) * p1) * 2 * 32 + lane;
        double y = 0.0, gg = 0.0;
        const int gf = g0 + q * g1;
        if (want_y0) {
          for (int ib = 0; ib < p1; ++ib) {
            y = fma(Lb[ib], src[(ib * 2) * 32], y);
            gg = fma(Lb[ib], src[(ib * 2 + 1) * 32], gg);
          }
          s.Y[(int64_t)(s.sf_face[rf] * s.Nqf + gf) * ne + e] = y;
        } else {
          for (int ib = 0; ib < p1; ++ib) gg = fma(Lb[ib], src[(ib * 2 + 1) * 32], gg);
        }
        s.Gy[(int64_t)(rf * s.Nqf + gf) * ne + e] = gg;
      }
    }
    return;
  }
  if (!live) return;
  // the rows the sweep computes (upwind and tangential points; every point
  // for shallow water): Gy in the sweep's slot order, and the element
  // values Y0 = Ey u^n there, which are all the initial trace reads (it
  // takes the upwind side, or both sides of a tangential point)
  const int nr = s.shared ? s.n_rows : s.nrows[e];
  for (int j = t; j < nr; j += kStepT) {
    const int r = s.shared ? s.rows[j] : s.rowid[j * ne + e];
    double y0 = 0.0, gy = 0.0;
    if (want_y0) {
      for (int k2 = 0; k2 < s.KE; ++k2) {
        const double wv = s.ey_val[r * s.KE + k2];
        const int i = s.ey_idx[r * s.KE + k2];
        y0 = fma(wv, s.u[i * ne + e], y0);
        gy = fma(wv, g[i * 32 + lane], gy);
      }
      s.Y[r * ne + e] = y0;
    } else {
      for (int k2 = 0; k2 < s.KE; ++k2)
        gy = fma(s.ey_val[r * s.KE + k2], g[s.ey_idx[r * s.KE + k2] * 32 + lane], gy);
    }
    s.Gy[j * ne + e] = gy;
  }
}

struct FinalParams {
  int64_t nel, nface;
  int n, NQFS, Nqf, F, shared, cn;
  const int32_t* elem_face;
  const double* uhat;           // [2][Nqf][nface]
  const IterState* it;
  const double* G;
  const double* H;
  double* u;
};

// Hsh: a shared operator H [n][NQFS]; uh: [NQFS][32] scratch; src: the trace
// the last sweep read.
__device__ __forceinline__ void final_tile(const FinalParams& p, const double* Hsh, double* uh,
                                           const double* src, int64_t tile) {
  const int lane = threadIdx.x, t = threadIdx.y;
  const int64_t ne = p.nel;
  const int64_t e = tile * 32 + lane;
  const bool live = e < ne;
  __syncthreads();
  if (live) {
    for (int f = 0; f < p.F; ++f) {
      const int64_t face = p.elem_face[f * ne + e];
      for (int g = t; g < p.Nqf; g += kStepT)
        uh[(f * p.Nqf + g) * 32 + lane] = src[g * p.nface + face];
    }
  }
  __syncthreads();
  if (!live) return;
  for (int r = t; r < p.n; r += kStepT) {
    double a0 = p.G[r * ne + e], a1 = 0.0;
    if (p.shared) {
      const double* Hr = Hsh + r * p.NQFS;
      int c = 0;
      for (; c + 1 < p.NQFS; c += 2) {
        a0 = fma(Hr[c], uh[c * 32 + lane], a0);
        a1 = fma(Hr[c + 1], uh[(c + 1) * 32 + lane], a1);
      }
      if (c < p.NQFS) a0 = fma(Hr[c], uh[c * 32 + lane], a0);
    } else {
      const double* Hr = p.H + (int64_t)r * p.NQFS * ne + e;
      int c = 0;
      for (; c + 1 < p.NQFS; c += 2) {
        a0 = fma(Hr[c * ne], uh[c * 32 + lane], a0);
        a1 = fma(Hr[(c + 1) * ne], uh[(c + 1) * 32 + lane], a1);
      }
      if (c < p.NQFS) a0 = fma(Hr[c * ne], uh[c * 32 + lane], a0);
    }
    double acc = a0 + a1;
    if (p.cn) acc = 2.0 * acc - p.u[r * ne + e];
    p.u[r * ne + e] = acc;
  }
}

// The transport trace at face point (gf, face): the trace formula (eq.
// transportLocale) from the element values Y at the point, with the exterior
// value g on boundary faces (Crank-Nicolson: the mean of the two levels'
// data); sgn = sgn(beta.n^-) at the point.
__device__ __forceinline__ double transport_trace_point(
    int64_t nel, int64_t nface, int Nqf, int cn, const int32_t* face_elem,
    const int8_t* face_local, const int8_t* sgn, const double* Y, const double* gb,
    const double* gb_old, int gf, int64_t face) {
  const int em = face_elem[face];
  const int ep = face_elem[nface + face];
  const int fm = face_local[face];
  const int fpl = face_local[nface + face];
  const int64_t pt = (int64_t)gf * nface + face;
  const int64_t ym_off = (int64_t)gf * nel;
  const int s = sgn[pt];
  double ext = 0.0;
  if (ep < 0) ext = cn ? 0.5 * (gb[pt] + gb_old[pt]) : gb[pt];
  if (s > 0) return Y[ym_off + (int64_t)fm * Nqf * nel + em];
  if (s < 0) return (ep >= 0) ? Y[ym_off + (int64_t)fpl * Nqf * nel + ep] : ext;
  const double ym = Y[ym_off + (int64_t)fm * Nqf * nel + em];
  const double yp = (ep >= 0) ? Y[ym_off + (int64_t)fpl * Nqf * nel + ep] : ext;
  return 0.5 * (ym + yp);
}

}  // namespace ehdg
