// CUDA kernels of libehdg (sm_103a): local-operator assembly and factorisation,
// the per-step right-hand side, the element sweep, the face trace update with
// its FP64 residual reduction, and the end-of-step reconstruction.
//
// Layout in HBM: per-element quantities are structure-of-arrays with the
// element index innermost ([row][elem] or [row][col][elem]) so that a warp of
// consecutive elements reads consecutive addresses; traces are [point][face].
#include <cuda_runtime.h>

#include <cmath>

#include "ehdg_internal.h"
#include "step_tiles.cuh"

namespace ehdg {

namespace {

// ---------------------------------------------------------------------------
// tensor-product basis evaluation from the 1D tables
// ---------------------------------------------------------------------------
__device__ __forceinline__ int digit(int v, int base, int k) {
  for (int i = 0; i < k; ++i) v /= base;
  return v % base;
}

// phi_i at volume quadrature point g
__device__ double vphi(const RefTables& R, int i, int g) {
  const int n1 = R.p + 1;
  double v = 1.0;
  for (int a = 0; a < R.dim; ++a) v *= R.L[digit(g, R.q, a) * kMaxP1 + digit(i, n1, a)];
  return v;
}

// d phi_i / d r_ax at volume point g
__device__ double vdphi(const RefTables& R, int ax, int i, int g) {
  const int n1 = R.p + 1;
  double v = 1.0;
  for (int a = 0; a < R.dim; ++a) {
    const int ga = digit(g, R.q, a), ia = digit(i, n1, a);
    v *= (a == ax) ? R.D[ga * kMaxP1 + ia] : R.L[ga * kMaxP1 + ia];
  }
  return v;
}

// phi_i at point gf of local face f (tangential axes increasing, first fastest)
__device__ double fphi(const RefTables& R, int f, int i, int gf) {
  const int n1 = R.p + 1;
  const int ax = f >> 1, side = f & 1;
  double v = R.Lend[side * kMaxP1 + digit(i, n1, ax)];
  int t = 0;
  for (int a = 0; a < R.dim; ++a) {
    if (a == ax) continue;
    v *= R.L[digit(gf, R.q, t) * kMaxP1 + digit(i, n1, a)];
    ++t;
  }
  return v;
}

__device__ double vweight(const RefTables& R, int g) {
  double w = 1.0;
  for (int a = 0; a < R.dim; ++a) w *= R.om[digit(g, R.q, a)];
  return w;
}

__device__ double fweight(const RefTables& R, int gf) {
  double w = 1.0;
  for (int t = 0; t < R.dim - 1; ++t) w *= R.om[digit(gf, R.q, t)];
  return w;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One full wave of resident blocks, capped by the number of tiles.
template <class K>
int persistent_grid(K kernel, int threads, size_t smem, int64_t ntiles) {
  fn_carveout((const void*)kernel);
  const int bpsm = fn_blocks_per_sm((const void*)kernel, threads, smem);
  int64_t g = (int64_t)bpsm * device_sms();
  if (g > ntiles) g = ntiles;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

// ===========================================================================
// Assembly + Gauss-Jordan: one CTA per element
// ===========================================================================
struct AsmParams {
  RefTables R;
  int pde, n, NQFS, KE;
  double tcoef;                 // coefficient of the mass term in A (1/dt_eff, 0 for steady)
  double Phi;
  double beta_c[3];
  double cor_f0, cor_beta, cor_ym, friction;   // shallow-water source terms
  int variable;
  const double* elem_h;         // [nel][dim]
  const double* elem_lo;        // [nel][dim] (beta-plane Coriolis), or null
  const double* beta_nodes;     // [nel][dim][Np]
  const int* ey_idx;
  const double* ey_val;
  double* P;
  double* H;
  double* Hy;
  // shared transport operator of hexahedra, sum-factorised sweep: the columns
  // of A^{-1} at the element's boundary nodes, Ab = A^{-1}[:, bnd] (n x NB),
  // and Dy = Ey A^{-1}[:, bnd] at every face point (NQFS x NB); null if unused
  int NB;
  const int* bnd;               // [NB] boundary node indices
  double* Ab;
  double* Dy;
  int64_t ne_out;               // element stride of the outputs (1 for a shared operator)
  int* err;
};

__global__ void k_assemble(const AsmParams a) {
  extern __shared__ double sm[];
  const RefTables& R = a.R;
  const int e = blockIdx.x;
  const int n = a.n, NQFS = a.NQFS, Np = R.Np, dim = R.dim, Nqf = R.Nqf;
  const int NB = a.Dy ? a.NB : 0;             // unit columns of the boundary nodes
  const int ncol = 2 * n + NQFS + NB;
  int Q = 1;
  for (int d = 0; d < dim; ++d) Q *= R.q;
  const int F = 2 * dim;

  double* aug = sm;                         // [n][ncol]
  double* bn = aug + n * ncol;              // [dim][Np]
  double* bq = bn + dim * Np;               // [dim][Q]
  double* dbq = bq + dim * Q;               // [dim][Q]
  double* bf = dbq + dim * Q;               // [F][Nqf] beta.n at face points
  double* fac = bf + F * Nqf;               // [n] elimination column
  __shared__ int piv;
  __shared__ double hsh[3];

  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid < dim) hsh[tid] = a.elem_h[(int64_t)e * dim + tid];
  for (int t = tid; t < dim * Np; t += nt) {
    const int ax = t / Np;
    bn[t] = a.variable ? a.beta_nodes[(int64_t)e * dim * Np + t] : a.beta_c[ax];
  }
  __syncthreads();
  double J = 1.0;
  for (int d = 0; d < dim; ++d) J *= 0.5 * hsh[d];

  if (a.pde == EHDG_TRANSPORT) {
    for (int t = tid; t < dim * Q; t += nt) {
      const int ax = t / Q, g = t % Q;
      double s = 0.0, ds = 0.0;
      for (int c = 0; c < Np; ++c) {
        s += vphi(R, c, g) * bn[ax * Np + c];
        ds += vdphi(R, ax, c, g) * bn[ax * Np + c];
      }
      bq[t] = s;
      dbq[t] = ds;
    }
    for (int t = tid; t < F * Nqf; t += nt) {
      const int f = t / Nqf, gf = t % Nqf, ax = f >> 1;
      double s = 0.0;
      for (int c = 0; c < Np; ++c) s += fphi(R, f, c, gf) * bn[ax * Np + c];
      bf[t] = (f & 1) ? s : -s;
    }
  }
  __syncthreads();

  // ---- fill [A | Mblk | B]
  if (a.pde == EHDG_TRANSPORT) {
    for (int t = tid; t < n * n; t += nt) {
      const int i = t / n, j = t % n;
      double m = 0.0, adv = 0.0;
      for (int g = 0; g < Q; ++g) {
        const double w = vweight(R, g) * J;
        const double pi = vphi(R, i, g), pj = vphi(R, j, g);
        double div = 0.0;
        for (int ax = 0; ax < dim; ++ax)
          div += (2.0 / hsh[ax]) * (dbq[ax * Q + g] * pi + bq[ax * Q + g] * vdphi(R, ax, i, g));
        m += w * pi * pj;
        adv -= w * pj * div;
      }
      double fc = 0.0;
      for (int f = 0; f < F; ++f) {
        const int ax = f >> 1;
        const double jf = J * 2.0 / hsh[ax];
        for (int gf = 0; gf < Nqf; ++gf) {
          const double b = bf[f * Nqf + gf];
          const double fi = fphi(R, f, i, gf);
          if (fi == 0.0) continue;
          fc += jf * fweight(R, gf) * (b + fabs(b)) * fi * fphi(R, f, j, gf);
        }
      }
      aug[i * ncol + j] = a.tcoef * m + adv + fc;
      aug[i * ncol + n + j] = m;
    }
    for (int t = tid; t < n * NQFS; t += nt) {
      const int i = t / NQFS, s = t % NQFS;
      const int f = s / Nqf, gf = s % Nqf, ax = f >> 1;
      const double jf = J * 2.0 / hsh[ax];
      aug[i * ncol + 2 * n + s] = jf * fweight(R, gf) * fabs(bf[s]) * fphi(R, f, i, gf);
    }
  } else {
    // linearised shallow water, unknowns (phi, u, v), Sec. 3 eq. localSolverDD
    const double Phi = a.Phi, sq = sqrt(Phi);
    for (int t = tid; t < n * n; t += nt) {
      const int I = t / n, Jc = t % n;
      const int fi = I / Np, i = I % Np, fj = Jc / Np, j = Jc % Np;
      double m = 0.0, mf = 0.0, gx[3] = {0.0, 0.0, 0.0};
      const double lo_y = a.elem_lo ? a.elem_lo[(int64_t)e * dim + 1] : 0.0;
      for (int g = 0; g < Q; ++g) {
        const double w = vweight(R, g) * J;
        const double pj = vphi(R, j, g);
        const double pij = vphi(R, i, g) * pj;
        m += w * pij;
        // Coriolis parameter f = f0 + beta (y - y_m) at the point's physical y
        const double y = lo_y + 0.5 * hsh[1] * (R.xi[digit(g, R.q, 1)] + 1.0);
        mf += w * (a.cor_f0 + a.cor_beta * (y - a.cor_ym)) * pij;
        for (int ax = 0; ax < dim; ++ax) gx[ax] += w * (2.0 / hsh[ax]) * vdphi(R, ax, i, g) * pj;
      }
      double ef[6];
      for (int f = 0; f < F; ++f) {
        const int ax = f >> 1;
        const double jf = J * 2.0 / hsh[ax];
        double s = 0.0;
        for (int gf = 0; gf < Nqf; ++gf) s += jf * fweight(R, gf) * fphi(R, f, i, gf) * fphi(R, f, j, gf);
        ef[f] = s;
      }
      double A = 0.0, Mb = 0.0;
      if (fi == 0 && fj == 0) {
        A = a.tcoef * m;
        for (int f = 0; f < F; ++f) A += sq * ef[f];
        Mb = m;
      } else if (fi == 0) {
        const int ax = fj - 1;
        A = -Phi * gx[ax];
        for (int f = 0; f < F; ++f)
          if ((f >> 1) == ax) A += Phi * ((f & 1) ? 1.0 : -1.0) * ef[f];
      } else if (fj == 0) {
        A = -Phi * gx[fi - 1];
      } else if (fi == fj) {
        // velocity rows: mass term and bottom friction (gamma Phi u, w)
        A = (a.tcoef + a.friction) * Phi * m;
        Mb = Phi * m;
      } else {
        // Coriolis: -(f Phi v, w) in the u-row, +(f Phi u, w) in the v-row
        A = (fi == 1 ? -1.0 : 1.0) * Phi * mf;
      }
      aug[I * ncol + Jc] = A;
      aug[I * ncol + n + Jc] = Mb;
    }
    for (int t = tid; t < n * NQFS; t += nt) {
      const int I = t / NQFS, s = t % NQFS;
      const int fi = I / Np, i = I % Np;
      const int f = s / Nqf, gf = s % Nqf, ax = f >> 1;
      const double jf = J * 2.0 / hsh[ax];
      const double base = jf * fweight(R, gf) * fphi(R, f, i, gf);
      double v = 0.0;
      if (fi == 0) v = sq * base;
      else if (fi - 1 == ax) v = -Phi * ((f & 1) ? 1.0 : -1.0) * base;
      aug[I * ncol + 2 * n + s] = v;
    }
  }
  // unit columns e_bnd[b] (sum-factorised sweep): they become A^{-1}[:, bnd]
  for (int t = tid; t < n * NB; t += nt) {
    const int i = t / NB, b = t % NB;
    aug[i * ncol + 2 * n + NQFS + b] = (a.bnd[b] == i) ? 1.0 : 0.0;
  }
  __syncthreads();

  // ---- Gauss-Jordan elimination with partial pivoting: [A|Mblk|B] -> [I|P|H]
  for (int k = 0; k < n; ++k) {
    if (tid < 32) {
      double best = -1.0;
      int bi = k;
      for (int r = k + tid; r < n; r += 32) {
        const double v = fabs(aug[r * ncol + k]);
        if (v > best) { best = v; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) piv = bi;
    }
    __syncthreads();
    if (piv != k) {
      for (int j = tid; j < ncol; j += nt) {
        const double tmp = aug[k * ncol + j];
        aug[k * ncol + j] = aug[piv * ncol + j];
        aug[piv * ncol + j] = tmp;
      }
      __syncthreads();
    }
    const double pv = aug[k * ncol + k];
    if (pv == 0.0 || !isfinite(pv)) {
      if (tid == 0) atomicExch(a.err, 1);
      return;   // uniform across the block: pv is read from shared memory
    }
    for (int r = tid; r < n; r += nt) fac[r] = aug[r * ncol + k];
    __syncthreads();
    const double inv = 1.0 / pv;
    for (int j = tid; j < ncol; j += nt) aug[k * ncol + j] *= inv;
    __syncthreads();
    for (int t = tid; t < n * ncol; t += nt) {
      const int r = t / ncol, j = t % ncol;
      if (r != k) aug[t] -= fac[r] * aug[k * ncol + j];
    }
    __syncthreads();
  }

  // ---- outputs: P = A^{-1} Mblk, H = A^{-1} B, Hy = Ey H
  const int64_t ne = a.ne_out;
  for (int t = tid; t < n * n; t += nt) {
    const int i = t / n, j = t % n;
    a.P[(int64_t)t * ne + e] = aug[i * ncol + n + j];
  }
  for (int t = tid; t < n * NQFS; t += nt) {
    const int i = t / NQFS, s = t % NQFS;
    a.H[(int64_t)t * ne + e] = aug[i * ncol + 2 * n + s];
  }
  for (int t = tid; t < NQFS * NQFS; t += nt) {
    const int s = t / NQFS, c = t % NQFS;
    double v = 0.0;
    for (int k = 0; k < a.KE; ++k) {
      const double ev = a.ey_val[s * a.KE + k];
      if (ev != 0.0) v += ev * aug[a.ey_idx[s * a.KE + k] * ncol + 2 * n + c];
    }
    a.Hy[(int64_t)t * ne + e] = v;
  }
  if (NB > 0) {   // shared operator only (ne = 1)
    const int c0 = 2 * n + NQFS;
    for (int t = tid; t < n * NB; t += nt) {
      const int i = t / NB, b = t % NB;
      a.Ab[t] = aug[i * ncol + c0 + b];
    }
    for (int t = tid; t < NQFS * NB; t += nt) {
      const int s = t / NB, b = t % NB;
      double v = 0.0;
      for (int k = 0; k < a.KE; ++k) {
        const double ev = a.ey_val[s * a.KE + k];
        if (ev != 0.0) v += ev * aug[a.ey_idx[s * a.KE + k] * ncol + c0 + b];
      }
      a.Dy[t] = v;
    }
  }
}

size_t asm_smem(const Ctx& c) {
  int Q = 1;
  for (int d = 0; d < c.dim; ++d) Q *= c.q;
  const int ncol = 2 * c.n + c.NQFS + (c.sf_Dy ? c.sf_NB : 0);
  return sizeof(double) * ((size_t)c.n * ncol + c.dim * c.Np + 2 * c.dim * Q + c.F * c.Nqf + c.n);
}

cudaError_t launch_assemble(Ctx& c, int n_assemble) {
  AsmParams a;
  a.R = c.ref;
  a.pde = c.pde;
  a.n = c.n;
  a.NQFS = c.NQFS;
  a.KE = c.KE;
  a.tcoef = (c.scheme == EHDG_STEADY) ? 0.0 : 1.0 / c.dt_eff;
  a.Phi = c.Phi;
  for (int d = 0; d < 3; ++d) a.beta_c[d] = c.beta_const[d];
  a.cor_f0 = c.cor_f0;
  a.cor_beta = c.cor_beta;
  a.cor_ym = c.cor_ym;
  a.friction = c.friction;
  a.elem_lo = c.elem_lo_d;
  a.variable = c.variable_beta ? 1 : 0;
  a.elem_h = c.geo.elem_h;
  a.beta_nodes = c.beta_nodes;
  a.ey_idx = c.ey_idx;
  a.ey_val = c.ey_val;
  a.P = c.P;
  a.H = c.H;
  a.Hy = c.Hy;
  a.NB = c.sf_NB;
  a.bnd = c.sf_bnd;
  a.Ab = c.sf_Ab;
  a.Dy = c.sf_Dy;
  a.ne_out = c.shared_op ? 1 : c.nel;
  a.err = reinterpret_cast<int*>(&c.it->status);
  const size_t smem = asm_smem(c);
  cudaError_t err = cudaFuncSetAttribute(k_assemble, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  k_assemble<<<n_assemble, 256, smem, c.stream>>>(a);
  return cudaGetLastError();
}

// ===========================================================================
// sgn(beta.n^-) at every face point (transport), from the minus element
// ===========================================================================
__global__ void k_face_signs(const RefTables R, Geometry geo, const double* beta_nodes,
                             int variable, double b0, double b1, double b2, int8_t* sgn) {
  const int64_t total = (int64_t)R.Nqf * geo.nface;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int gf = (int)(t / geo.nface);
    const int64_t face = t % geo.nface;
    const int em = geo.face_elem[face];
    const int f = geo.face_local[face];
    const int ax = f >> 1;
    double s = 0.0;
    if (variable) {
      const double* bn = beta_nodes + ((int64_t)em * R.dim + ax) * R.Np;
      for (int c = 0; c < R.Np; ++c) s += fphi(R, f, c, gf) * bn[c];
    } else {
      const double bc = ax == 0 ? b0 : (ax == 1 ? b1 : b2);
      for (int c = 0; c < R.Np; ++c) s += fphi(R, f, c, gf) * bc;
    }
    const double b = (f & 1) ? s : -s;
    sgn[t] = (int8_t)((b > 0.0) - (b < 0.0));
  }
}

cudaError_t launch_face_signs(Ctx& c) {
  const int64_t total = (int64_t)c.Nqf * c.nface;
  const int bs = 256;
  const int grid = (int)((total + bs - 1) / bs);
  k_face_signs<<<grid, bs, 0, c.stream>>>(c.ref, c.geo, c.beta_nodes, c.variable_beta ? 1 : 0,
                                           c.beta_const[0], c.beta_const[1], c.beta_const[2],
                                           c.sgn);
  return cudaGetLastError();
}

// ===========================================================================
// Per-step right-hand side: G = P w, Gy = Ey G, Y0 = Ey u^n
//   w = u^n / dt_eff + f (time-dependent) or w = f (steady)
// ===========================================================================
// Tile of 32 consecutive elements (threadIdx.x) x kStepT row groups
// (threadIdx.y); persistent over tiles. w and G of the tile live in shared
// memory; a shared operator P is staged once per block. The tile body is in
// step_tiles.cuh (the batched loop runs it too).
__global__ void __launch_bounds__(32 * kStepT) k_step(const __grid_constant__ StepParams s) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x, t = threadIdx.y, tid = t * 32 + lane;
  const int n = s.n;
  double* Psh = sm;                                   // n*n if shared
  double* w = sm + (s.shared ? n * n : 0);            // [n][32]
  double* g = w + n * 32;                             // [n][32]
  double* sfw = g + n * 32;                           // face passes (sf_ey)
  if (s.shared)
    for (int i = tid; i < n * n; i += 32 * kStepT) Psh[i] = s.P[i];
  const int64_t ntiles = (s.nel + 31) / 32;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
    step_tile(s, Psh, w, g, sfw, tile);
}

// The sum-factorised face-point pass of the step (hexahedra, one shared
// transport operator, sweep rows that are whole faces in face order, q = p+1):
// the row faces and their node grids. Returns false where it does not apply.
static bool step_sf_plan(const Ctx& c, StepParams& s) {
  s.sf_ey = 0;
  if (c.dim != 3 || !c.shared_op || c.pde != EHDG_TRANSPORT || c.q != c.p + 1 || c.p + 1 > 4)
    return false;
  if (c.n_rows % c.Nqf != 0 || (int)c.rows_host.size() != c.n_rows) return false;
  const int nf = c.n_rows / c.Nqf;
  if (nf < 1 || nf > 3) return false;
  const int p1 = c.p + 1;
  const int stride[3] = {1, p1, p1 * p1};
  for (int rf = 0; rf < nf; ++rf) {
    const int f = c.rows_host[rf * c.Nqf] / c.Nqf;
    for (int gf = 0; gf < c.Nqf; ++gf)
      if (c.rows_host[rf * c.Nqf + gf] != f * c.Nqf + gf) return false;
    const int ax = f >> 1, side = f & 1;
    const int ta = ax == 0 ? 1 : 0, tb = ax == 2 ? 1 : 2;   // tangential axes, a < b
    s.sf_face[rf] = f;
    s.sf_base[rf] = (side ? c.p : 0) * stride[ax];
    s.sf_sa[rf] = stride[ta];
    s.sf_sb[rf] = stride[tb];
  }
  for (int g = 0; g < c.q; ++g)
    for (int i = 0; i < p1; ++i) s.sfL[g * p1 + i] = c.r1d.L[g * p1 + i];
  s.sf_nf = nf;
  s.sf_p1 = p1;
  s.Nqf = c.Nqf;
  s.sf_ey = 1;
  return true;
}

cudaError_t launch_step(Ctx& c) {
  StepParams s;
  s.nel = c.nel;
  s.n = c.n;
  s.NQFS = c.NQFS;
  s.KE = c.KE;
  s.shared = c.shared_op ? 1 : 0;
  s.ucoef = (c.scheme == EHDG_STEADY) ? 0.0 : 1.0 / c.dt_eff;
  s.have_force = c.have_force ? 1 : 0;
  s.force_avg = (c.scheme == EHDG_CN) ? 1 : 0;
  s.P = c.P;
  s.u = c.u;
  s.force = c.force;
  s.force_old = c.force_old;
  s.ey_idx = c.ey_idx;
  s.ey_val = c.ey_val;
  s.rows = c.rows;
  s.n_rows = c.n_rows;
  s.rowid = c.rowid;
  s.nrows = c.nrows;
  s.G = c.G;
  s.Gy = c.Gy;
  s.Y = c.Y;
  s.warm = c.warm_ok ? c.warm : nullptr;
  s.g_ready = 0;
  s.sf_ey = 0;
  if (c.use_ozaki && c.oz_step.img) {
    cudaError_t e = launch_step_ozaki(c);
    if (e != cudaSuccess) return e;
    s.g_ready = 1;
  }
  step_sf_plan(c, s);
  const size_t smem =
      sizeof(double) * ((s.shared ? (size_t)c.n * c.n : 0) + 2 * (size_t)c.n * 32 +
                        (s.sf_ey ? (size_t)s.sf_nf * s.sf_p1 * s.sf_p1 * 2 * 32 : 0));
  cudaError_t err = fn_smem((const void*)k_step, smem);
  if (err != cudaSuccess) return err;
  const int grid = persistent_grid(k_step, 32 * kStepT, smem, (c.nel + 31) / 32);
  k_step<<<grid, dim3(32, kStepT), smem, c.stream>>>(s);
  return cudaGetLastError();
}

// ===========================================================================
// Element sweep (eq. transportLocalk1 / localSolverDD): Y = Gy + Hy uhat
//
// Block = 32 consecutive elements (threadIdx.x) x kElemT row groups
// (threadIdx.y): a warp reads one slot of 32 consecutive elements, i.e. a
// contiguous 256-byte segment of the [slot][col][elem] operator. Only the
// face-point rows the trace formula will read are computed: for a constant
// velocity the upwind/tangential faces (a list shared by all elements), for a
// per-node velocity each element's own compacted list (rowid/nrows).
// ===========================================================================
constexpr int kElemT = 4;

struct ElemParams {
  int64_t nel, nface;
  int NQFS, Nqf, F, shared, n_rows;
  const int* rows;              // shared operator: output rows
  const uint8_t* rowid;         // per-element operator: [slot][nel] row of a slot
  const uint8_t* nrows;         // [nel]
  const int32_t* elem_face;     // [F][nel]
  const double* uhat;           // [2][Nqf][nface] ping-pong pair, iteration k reads slot k&1
  const IterState* it;
  const double* Gy;             // [slot][nel]
  const double* Hy;             // shared: [NQFS][NQFS]; per element: [slot][NQFS][nel]
  double* Y;                    // [NQFS][nel]
};

template <int NQ>
__global__ void __launch_bounds__(32 * kElemT) k_elem(const ElemParams p) {
  extern __shared__ double sm[];
  const int nq = NQ > 0 ? NQ : p.NQFS;
  const int lane = threadIdx.x, t = threadIdx.y;
  double* Hsh = sm;
  double* uh = sm + (p.shared ? nq * nq : 0);          // [nq][32]
  if (p.shared)
    for (int i = t * 32 + lane; i < nq * nq; i += 32 * kElemT) Hsh[i] = p.Hy[i];
  const int64_t ne = p.nel;
  const int64_t e = blockIdx.x * 32LL + lane;
  const double* src = p.uhat + (int64_t)(p.it->k & 1) * p.Nqf * p.nface;
  if (e < ne) {
    for (int i = t; i < nq; i += kElemT) {
      const int f = i / p.Nqf, g = i - f * p.Nqf;
      const int64_t face = p.elem_face[f * ne + e];
      uh[i * 32 + lane] = src[g * p.nface + face];
    }
  }
  __syncthreads();
  if (e >= ne) return;
  const int nr = p.shared ? p.n_rows : p.nrows[e];
  for (int j = t; j < nr; j += kElemT) {
    double acc = p.Gy[j * ne + e];
    int r;
    if (p.shared) {
      r = p.rows[j];
      const double* Hr = Hsh + r * nq;
      if constexpr (NQ > 0) {
#pragma unroll
        for (int c = 0; c < NQ; ++c) acc += Hr[c] * uh[c * 32 + lane];
      } else {
        for (int c = 0; c < nq; ++c) acc += Hr[c] * uh[c * 32 + lane];
      }
    } else {
      r = p.rowid[j * ne + e];
      const double* Hr = p.Hy + (int64_t)j * nq * ne + e;
      if constexpr (NQ > 0) {
#pragma unroll
        for (int c = 0; c < NQ; ++c) acc += Hr[c * ne] * uh[c * 32 + lane];
      } else {
        for (int c = 0; c < nq; ++c) acc += Hr[c * ne] * uh[c * 32 + lane];
      }
    }
    p.Y[(int64_t)r * ne + e] = acc;
  }
}

template <int NQ>
static cudaError_t launch_elem_t(const ElemParams& p, size_t smem, int grid, cudaStream_t s) {
  cudaError_t err = fn_smem((const void*)k_elem<NQ>, smem);
  if (err != cudaSuccess) return err;
  k_elem<NQ><<<grid, dim3(32, kElemT), smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_elem(Ctx& c) {
  if (c.use_ozaki) return launch_elem_ozaki(c);
  ElemParams p;
  p.nel = c.nel;
  p.nface = c.nface;
  p.NQFS = c.NQFS;
  p.Nqf = c.Nqf;
  p.F = c.F;
  p.shared = c.shared_op ? 1 : 0;
  p.n_rows = c.n_rows;
  p.rows = c.rows;
  p.rowid = c.rowid;
  p.nrows = c.nrows;
  p.elem_face = c.geo.elem_face;
  p.uhat = c.uhat;
  p.it = c.it;
  p.Gy = c.Gy;
  p.Hy = c.Hy;
  p.Y = c.Y;
  const size_t smem = sizeof(double) * ((p.shared ? (size_t)c.NQFS * c.NQFS : 0) + (size_t)c.NQFS * 32);
  const int grid = (int)((c.nel + 31) / 32);
  switch (c.NQFS) {
    case 8: return launch_elem_t<8>(p, smem, grid, c.stream);
    case 12: return launch_elem_t<12>(p, smem, grid, c.stream);
    case 16: return launch_elem_t<16>(p, smem, grid, c.stream);
    case 20: return launch_elem_t<20>(p, smem, grid, c.stream);
    case 24: return launch_elem_t<24>(p, smem, grid, c.stream);
    case 28: return launch_elem_t<28>(p, smem, grid, c.stream);
    case 36: return launch_elem_t<36>(p, smem, grid, c.stream);
    case 40: return launch_elem_t<40>(p, smem, grid, c.stream);
    case 54: return launch_elem_t<54>(p, smem, grid, c.stream);
    case 96: return launch_elem_t<96>(p, smem, grid, c.stream);
    default: return launch_elem_t<0>(p, smem, grid, c.stream);
  }
}

// Per-element operator: the rows each element's sweep must produce (the face
// points where it is the upwind or tangential side, from the same sgn array
// the trace kernel uses; every point for shallow water), compacted into slots.
__global__ void k_rows(int64_t nel, int NQFS, int Nqf, int F, int transport,
                       const int32_t* elem_face, const int32_t* face_elem, int64_t nface,
                       const int8_t* sgn, uint8_t* rowid, uint8_t* nrows, uint8_t* nup) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nel) return;
  int j = 0;
  // pass 0: strictly upwind points (this element owns them); pass 1: beta.n = 0
  for (int pass = 0; pass < (transport ? 2 : 1); ++pass) {
    for (int s = 0; s < NQFS; ++s) {
      bool need = true;
      if (transport) {
        const int f = s / Nqf, g = s - f * Nqf;
        const int64_t face = elem_face[f * nel + e];
        const bool minus = face_elem[face] == (int32_t)e;
        const int sg = sgn[g * nface + face];
        const int own = minus ? sg : -sg;          // sgn(beta.n) seen from this element
        need = (pass == 0) ? (own > 0) : (own == 0);
      }
      if (need) rowid[(int64_t)(j++) * nel + e] = (uint8_t)s;
    }
    if (pass == 0) nup[e] = (uint8_t)j;
  }
  nrows[e] = (uint8_t)j;
}

// Move each element's needed rows of Hy to the front (slot order), in place:
// slot j takes row rowid[j] >= j, and no later slot reads a row below it.
__global__ void k_compact_hy(int64_t nel, int NQFS, const uint8_t* rowid, const uint8_t* nrows,
                             double* Hy) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nel) return;
  const int nr = nrows[e];
  for (int j = 0; j < nr; ++j) {
    const int r = rowid[(int64_t)j * nel + e];
    if (r == j) continue;
    for (int c = 0; c < NQFS; ++c)
      Hy[((int64_t)j * NQFS + c) * nel + e] = Hy[((int64_t)r * NQFS + c) * nel + e];
  }
}

cudaError_t launch_rows(Ctx& c) {
  const int grid = (int)((c.nel + 255) / 256);
  k_rows<<<grid, 256, 0, c.stream>>>(c.nel, c.NQFS, c.Nqf, c.F, c.pde == EHDG_TRANSPORT ? 1 : 0,
                                     c.geo.elem_face, c.geo.face_elem, c.nface, c.sgn, c.rowid,
                                     c.nrows, c.nup);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_compact_hy<<<grid, 256, 0, c.stream>>>(c.nel, c.NQFS, c.rowid, c.nrows, c.Hy);
  return cudaGetLastError();
}

// ===========================================================================
// Face trace update (eq. transportLocale; shallow-water trace) + residual
// ===========================================================================
struct FaceParams {
  Geometry geo;
  int pde, mode, cn, Nqf;
  double tol, res_scale;
  int max_iter;
  double fw[kMaxQ * kMaxQ];     // face Gauss weight of each face point (tangential product)
  const int8_t* sgn;
  const double* Y;              // [NQFS][nel]
  const double* gb;             // [Nqf][nface]
  const double* gb_old;
  double* uhat;                 // [2][Nqf][nface] ping-pong pair
  float* R_out;                 // mixed precision: F(uhat) - uhat (or null)
  double* partials;
  IterState* it;
  double* hist;
  int graph_mode;               // set the while-node condition from the last block
  cudaGraphConditionalHandle handle;
  const int* warm;              // initial mode: warm start flag (or null)
};

constexpr int kFaceBlock = 256;
// one wave: 4 resident 256-thread blocks per SM; each thread strides over
// several faces, so the reduction's adds are spread over more points
constexpr int kFaceMaxBlocks = 608;

// Grid: x strides over faces, y = face point. Block partials are reduced in a
// fixed order by the last block to finish (deterministic).
__global__ void __launch_bounds__(kFaceBlock) k_face(const FaceParams p) {
  __shared__ double red[kFaceBlock / 32];
  __shared__ bool last;
  const int64_t nface = p.geo.nface, nel = p.geo.nel;
  const int64_t total = (int64_t)p.Nqf * nface;
  const int gf = blockIdx.y;
  // every block reads the counter before the last block advances it
  const int kk = (p.mode == kFaceIterate) ? p.it->k : 0;
  const double* uh_old = p.uhat + (int64_t)(kk & 1) * total + (int64_t)gf * nface;
  double* uh_new = p.uhat + (int64_t)((p.mode == kFaceIterate ? kk + 1 : 0) & 1) * total +
                   (int64_t)gf * nface;
  const double wg = p.fw[gf];
  const int64_t ym_off = (int64_t)gf * nel;   // + (local face * Nqf) * nel + elem
  // warm start: slot 0 holds the previous step's final trace, the trace
  // formula of u^n at every point but the inflow boundary ones, which
  // k_trace0_warm sets (every other point of slot 1 is written by the first
  // sweep before any sweep reads it)
  if (p.mode != kFaceIterate && p.warm && *p.warm) return;
  double acc = 0.0;
  for (int64_t face = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; face < nface;
       face += (int64_t)gridDim.x * blockDim.x) {
    const int em = p.geo.face_elem[face];
    const int ep = p.geo.face_elem[nface + face];
    const int fm = p.geo.face_local[face];
    const int fpl = p.geo.face_local[nface + face];
    double uh;
    if (p.pde == EHDG_TRANSPORT) {
      uh = transport_trace_point(nel, nface, p.Nqf, p.cn, p.geo.face_elem, p.geo.face_local,
                                 p.sgn, p.Y, p.gb, p.gb_old, gf, face);
    } else {
      const double ym = p.Y[ym_off + (int64_t)fm * p.Nqf * nel + em];
      uh = (ep >= 0) ? ym + p.Y[ym_off + (int64_t)fpl * p.Nqf * nel + ep] : 2.0 * ym;
    }
    if (p.mode == kFaceIterate) {
      // the point weight wg is the block's; it multiplies the sum once below
      const double d = uh - uh_old[face];
      acc = fma(p.geo.face_jf[face] * d, d, acc);
      if (p.R_out) p.R_out[(int64_t)gf * nface + face] = (float)d;
    } else {
      uh_new[total + face] = uh;     // both slots: points no sweep rewrites keep this value
    }
    uh_new[face] = uh;
  }
  if (p.mode != kFaceIterate) return;

  // deterministic reduction: warp -> block -> partials[block] -> last block
  const unsigned int nblocks = gridDim.x * gridDim.y;
  const unsigned int bid = blockIdx.y * gridDim.x + blockIdx.x;
  acc = warp_sum(acc * wg);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (wid == 0) {
    double v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) {
      p.partials[bid] = v;
      __threadfence();
      const unsigned int ticket = atomicAdd(&p.it->counter, 1u);
      last = (ticket == nblocks - 1);
    }
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v = 0.0;
  for (unsigned int i = threadIdx.x; i < nblocks; i += blockDim.x)
    v += reinterpret_cast<volatile double*>(p.partials)[i];
  v = warp_sum(v);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
    const double r = p.res_scale * sqrt(sum);
    IterState* it = p.it;
    const int k = it->k;
    if (k < p.max_iter) p.hist[k] = r;
    it->k = k + 1;
    it->r_last = r;
    it->counter = 0u;
    int cont = 1, status = EHDG_OK;
    if (!isfinite(r)) { cont = 0; status = EHDG_ERR_DIVERGED; }
    else if (r < p.tol) { cont = 0; status = EHDG_OK; }
    else if (k + 1 >= p.max_iter) { cont = 0; status = EHDG_ERR_NOT_CONVERGED; }
    it->cont = cont;
    it->status = status;
    __threadfence();
    if (p.graph_mode) cudaGraphSetConditional(p.handle, (unsigned int)cont);
  }
}

int face_grid_x(int64_t nface, int Nqf) {
  int64_t gx = (nface + kFaceBlock - 1) / kFaceBlock;
  int64_t cap = kFaceMaxBlocks / Nqf;
  if (cap < 1) cap = 1;
  if (gx > cap) gx = cap;
  return gx < 1 ? 1 : (int)gx;
}

// Warm-start initial trace: the inflow boundary points (beta.n < 0 seen from
// the inside; no point has beta.n = 0 where the warm start is on) take the
// new step's boundary data in both slots. Nothing to do on a cold start.
__global__ void k_trace0_warm(const int* warm, const int32_t* bface, int64_t n_bface, int Nqf,
                              int64_t nface, const int8_t* sgn, const double* gb, double* uhat) {
  if (!*warm) return;
  const int64_t total = (int64_t)Nqf * nface;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_bface * Nqf;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / Nqf;
    const int g = (int)(t - b * Nqf);
    const int64_t pt = (int64_t)g * nface + bface[b];
    if (sgn[pt] < 0) {
      uhat[pt] = gb[pt];
      uhat[total + pt] = gb[pt];
    }
  }
}

int face_launches(const Ctx& c, int mode) {
  // transport: the warm start's inflow boundary points (shallow water has none)
  return (mode == kFaceInitial && c.warm_ok && c.pde == EHDG_TRANSPORT && c.n_bface > 0) ? 2 : 1;
}

cudaError_t launch_face(Ctx& c, int mode, int graph_mode) {
  FaceParams p;
  p.graph_mode = graph_mode;
  p.handle = c.handle;
  p.geo = c.geo;
  p.pde = c.pde;
  p.mode = mode;
  p.warm = c.warm_ok ? c.warm : nullptr;
  p.cn = (c.scheme == EHDG_CN) ? 1 : 0;
  p.Nqf = c.Nqf;
  p.tol = c.tol;
  p.res_scale = c.res_scale;
  p.max_iter = c.max_iter;
  for (int g = 0; g < c.Nqf; ++g) {
    double w = 1.0;
    int rem = g;
    for (int t = 0; t < c.dim - 1; ++t) {
      w *= c.r1d.om[rem % c.q];
      rem /= c.q;
    }
    p.fw[g] = w;
  }
  p.sgn = c.sgn;
  p.Y = c.Y;
  p.gb = c.gb;
  p.gb_old = c.gb_old;
  p.uhat = c.uhat;
  p.R_out = c.mixed ? c.R32 : nullptr;
  p.partials = c.partials;
  p.it = c.it;
  p.hist = c.hist;
  const dim3 grid(face_grid_x(c.nface, c.Nqf), c.Nqf);
  k_face<<<grid, kFaceBlock, 0, c.stream>>>(p);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess || face_launches(c, mode) < 2) return err;
  const int64_t nb = c.n_bface * c.Nqf;
  const int g2 = (int)std::min<int64_t>((nb + 255) / 256, 152 * 8);
  k_trace0_warm<<<g2, 256, 0, c.stream>>>(c.warm, c.bface, c.n_bface, c.Nqf, c.nface, c.sgn,
                                           c.gb, c.uhat);
  return cudaGetLastError();
}

// ===========================================================================
// End of step: u^{n+1} = G + H uhat (Crank-Nicolson: 2 v - u^n), trace update
// ===========================================================================
__global__ void __launch_bounds__(32 * kStepT) k_final(const FinalParams p) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x, t = threadIdx.y, tid = t * 32 + lane;
  double* Hsh = sm;
  double* uh = sm + (p.shared ? p.n * p.NQFS : 0);     // [NQFS][32]
  if (p.shared)
    for (int i = tid; i < p.n * p.NQFS; i += 32 * kStepT) Hsh[i] = p.H[i];
  const int64_t ntiles = (p.nel + 31) / 32;
  // Algorithm 1 returns u^{k+1}, the local solve with the trace uhat^k
  const double* src = p.uhat + (int64_t)((p.it->k + 1) & 1) * p.Nqf * p.nface;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
    final_tile(p, Hsh, uh, src, tile);
}

// The final trace uhat^{K} (slot K&1) becomes the state's trace in slot 0
// (Crank-Nicolson: 2 vhat - uhat^n, and the previous-level copies uhat^n and
// g_old are updated; backward Euler and steady solves read neither, and
// with K even the final trace is in slot 0 already).
__global__ void k_trace_end(int64_t total, int cn, const IterState* it, double* uhat,
                            double* uhat_n, const double* gb, double* gb_old, int* warm) {
  const double* fin = uhat + (int64_t)(it->k & 1) * total;
  // at least one sweep ran: its owned outputs are Ey of the reconstruction
  if (warm && blockIdx.x == 0 && threadIdx.x == 0) *warm = it->k >= 1 ? 1 : 0;
  if (!cn && !(it->k & 1)) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (!cn) {
      uhat[t] = fin[t];
      continue;
    }
    const double v = 2.0 * fin[t] - uhat_n[t];
    uhat[t] = v;
    uhat_n[t] = v;
    gb_old[t] = gb[t];
  }
}

cudaError_t launch_final(Ctx& c) {
  FinalParams p;
  p.nel = c.nel;
  p.nface = c.nface;
  p.n = c.n;
  p.NQFS = c.NQFS;
  p.Nqf = c.Nqf;
  p.F = c.F;
  p.shared = c.shared_op ? 1 : 0;
  p.cn = (c.scheme == EHDG_CN) ? 1 : 0;
  p.elem_face = c.geo.elem_face;
  p.uhat = c.uhat;
  p.it = c.it;
  p.G = c.G;
  p.H = c.H;
  p.u = c.u;
  cudaError_t err;
  if (c.use_ozaki && c.oz_final.img) {
    err = launch_final_ozaki(c);
  } else if (c.Ht) {
    err = launch_final_tiled(c);
  } else if (c.use_sf) {
    err = launch_final_sf(c);
  } else {
    const size_t smem =
        sizeof(double) * ((p.shared ? (size_t)c.n * c.NQFS : 0) + (size_t)c.NQFS * 32);
    err = fn_smem((const void*)k_final, smem);
    if (err != cudaSuccess) return err;
    const int grid = persistent_grid(k_final, 32 * kStepT, smem, (c.nel + 31) / 32);
    k_final<<<grid, dim3(32, kStepT), smem, c.stream>>>(p);
    err = cudaGetLastError();
  }
  if (err != cudaSuccess) return err;
  const int64_t total = (int64_t)c.Nqf * c.nface;
  k_trace_end<<<(int)((total + 255) / 256), 256, 0, c.stream>>>(
      total, p.cn, c.it, c.uhat, c.uhat_n, c.gb, c.gb_old, c.warm_ok ? c.warm : nullptr);
  return cudaGetLastError();
}

// ===========================================================================
// misc: Y = Ey u (initial trace input), transposes, iteration reset
// ===========================================================================
__global__ void k_extract(int64_t nel, int NQFS, int KE, const int* ey_idx, const double* ey_val,
                          const double* u, double* Y) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nel) return;
  for (int r = 0; r < NQFS; ++r) {
    double y = 0.0;
    for (int k = 0; k < KE; ++k) y += ey_val[r * KE + k] * u[(int64_t)ey_idx[r * KE + k] * nel + e];
    Y[(int64_t)r * nel + e] = y;
  }
}

cudaError_t launch_extract(Ctx& c) {
  k_extract<<<(int)((c.nel + 127) / 128), 128, 0, c.stream>>>(c.nel, c.NQFS, c.KE, c.ey_idx,
                                                                c.ey_val, c.u, c.Y);
  return cudaGetLastError();
}

// src [rows][cols] -> dst [cols][rows], 32x32 tiles on a 1D grid of tiles
__global__ void k_transpose(const double* __restrict__ src, double* __restrict__ dst,
                            int64_t rows, int64_t cols, int64_t ntc) {
  __shared__ double tile[32][33];
  const int64_t tr = blockIdx.x / ntc, tc = blockIdx.x % ntc;
  const int64_t c0 = tc * 32, r0 = tr * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = r0 + k, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = src[r * cols + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t c = c0 + k, r = r0 + threadIdx.x;
    if (r < rows && c < cols) dst[c * rows + r] = tile[threadIdx.x][k];
  }
}

static cudaError_t transpose(const double* src, double* dst, int64_t rows, int64_t cols,
                             cudaStream_t s) {
  if (rows == 0 || cols == 0) return cudaSuccess;
  const int64_t ntr = (rows + 31) / 32, ntc = (cols + 31) / 32;
  if (ntr * ntc > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_transpose<<<(unsigned)(ntr * ntc), dim3(32, 8), 0, s>>>(src, dst, rows, cols, ntc);
  return cudaGetLastError();
}

cudaError_t launch_aos_to_soa(const double* src, double* dst, int64_t outer, int inner,
                              cudaStream_t s) {
  return transpose(src, dst, outer, inner, s);
}

cudaError_t launch_soa_to_aos(const double* src, double* dst, int64_t outer, int inner,
                              cudaStream_t s) {
  return transpose(src, dst, inner, outer, s);
}

// Boundary data of the boundary faces only: src [n_face][Nqf] (device memory,
// or pinned host memory through its device mapping), dst [Nqf][n_face]. A
// warp reads consecutive points of one face row, so each face's Nqf values
// come as one contiguous read.
__global__ void k_gather_boundary(const double* __restrict__ src, const int32_t* bface,
                                  int64_t n_b, int Nqf, int64_t nface, double* dst) {
  const int64_t total = n_b * Nqf;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / Nqf;
    const int g = (int)(t - b * Nqf);
    const int64_t f = bface[b];
    dst[(int64_t)g * nface + f] = src[f * Nqf + g];
  }
}

cudaError_t launch_gather_boundary(const Ctx& c, const double* src, double* dst) {
  const int64_t total = c.n_bface * c.Nqf;
  if (total == 0) return cudaSuccess;
  int64_t grid = (total + 255) / 256;
  if (grid > 152 * 16) grid = 152 * 16;
  k_gather_boundary<<<(unsigned)grid, 256, 0, c.stream>>>(src, c.bface, c.n_bface, c.Nqf,
                                                          c.nface, dst);
  return cudaGetLastError();
}

// Per-step bookkeeping after the end-of-step kernels: iterations and status
// of step it->step, then advance the step counter.
__global__ void k_step_end(IterState* it, int* iters, int* status, int cap) {
  const int s = it->step;
  if (s >= 0 && s < cap) {
    iters[s] = it->k;
    status[s] = it->status;
  }
  it->step = s + 1;
}

cudaError_t launch_step_end(Ctx& c) {
  k_step_end<<<1, 1, 0, c.stream>>>(c.it, c.step_iters, c.step_status, c.step_cap);
  return cudaGetLastError();
}

// Per-instance device time of a batched step: %globaltimer at the start of
// the instance's branch, and the elapsed time added at its end.
__global__ void k_stamp(unsigned long long* t_start, unsigned long long* t_acc, int i, int end) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  if (end) t_acc[i] += t - t_start[i];
  else t_start[i] = t;
}

cudaError_t launch_stamp(cudaStream_t s, unsigned long long* t_start, unsigned long long* t_acc,
                         int i, int end) {
  k_stamp<<<1, 1, 0, s>>>(t_start, t_acc, i, end);
  return cudaGetLastError();
}

__global__ void k_reset(IterState* it) {
  it->k = 0;
  it->cont = 1;
  it->status = EHDG_OK;
  it->counter = 0u;
  it->bar = 0u;
  it->abort = 0;
  it->r_last = 0.0;
}

cudaError_t launch_reset_iter(Ctx& c) {
  k_reset<<<1, 1, 0, c.stream>>>(c.it);
  return cudaGetLastError();
}

}  // namespace ehdg
