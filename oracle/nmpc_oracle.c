/* Oracle for the parametric interior-point NMPC hot path -- TEST INFRASTRUCTURE.
 *
 * Plain FP64 CPU code written from arXiv 2606.04725 (Sec. 3.2, Algorithm 2)
 * and the interior-point method it builds on (Wachter & Biegler 2006, cited by
 * the paper for the Newton system, inertia correction and termination test).
 * Only tests, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it.
 * It shares no code with the CUDA library.
 *
 * Linear algebra: the condensed Lifted-KKT matrix is assembled as a symmetric
 * band matrix in the natural stage order and factored by a textbook banded
 * Cholesky (no reordering, no supernodes).  Success of the Cholesky is the
 * inertia test of eq. (infiniteOCP-inertia).  With options.linsolve = 1 the
 * same matrix goes to a plain sparse Cholesky after a nested-dissection
 * ordering of the oracle's own (or_sparse.inc), for plates whose band is too
 * wide; the arithmetic per entry and the pivot test are the same.
 *
 * HyKKT form (options.kkt = 1), the alternative to Lifted-KKT that Sec. 3.2.2
 * names, after the hybrid direct-iterative method it cites (Regev et al.
 * 2023; Golub & Greif 2003): the equalities stay with multipliers lambda, the
 * augmented matrix W + Sigma_y + delta_w I + gamma H^T H takes the same band
 * Cholesky (and its success the same inertia test), and conjugate gradients on
 * the Schur complement give lambda's step.
 */
#include "nmpc_oracle.h"

#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- layout */

static int or_off_x(const or_problem* p, int k) { return k == 0 ? 0 : p->nx + (k - 1) * (p->nx + p->nu); }
static int or_off_u(const or_problem* p, int k) { return or_off_x(p, k) + p->nx; }

/* actuator segments touching the boundary faces of plate cell c, ascending.
 * Sides: 0 bottom (j = 0), 1 right (i = g-1), 2 top (j = g-1), 3 left (i = 0);
 * each side carries S/4 segments of g/(S/4) cells. */
static int or_plate_cell_segments(const or_problem* p, int c, int* segs) {
  const int g = p->g, per = p->S / 4, len = g / per;
  const int i = c % g, j = c / g;
  int k = 0;
  if (j == 0) segs[k++] = 0 * per + i / len;
  if (i == g - 1) segs[k++] = 1 * per + j / len;
  if (j == g - 1) segs[k++] = 2 * per + i / len;
  if (i == 0) segs[k++] = 3 * per + j / len;
  if (k == 2 && segs[0] > segs[1]) { int t = segs[0]; segs[0] = segs[1]; segs[1] = t; }
  return k;
}

/* ------------------------------------------- model code, real and complex */

#define R double
#define SFX(name) name##_d
#define SIN sin
#define COS cos
#define CBRT cbrt
#define SQRT sqrt
#include "or_model.inc"
#undef R
#undef SFX
#undef SIN
#undef COS
#undef CBRT
#undef SQRT

#define R double complex
#define SFX(name) name##_z
#define SIN csin
#define COS ccos
#define CBRT(z) cpow((z), 1.0 / 3.0)
#define SQRT csqrt
#include "or_model.inc"
#undef R
#undef SFX
#undef SIN
#undef COS
#undef CBRT
#undef SQRT

int or_setup(or_problem* p) {
  if (p->model == OR_DISTILL) { p->nx = p->N; p->nu = 1; }
  else if (p->model == OR_PLATE) {
    if (p->g < 2 || p->S < 4 || p->S % 4 || p->g % (p->S / 4)) return -1;
    p->nx = p->g * p->g; p->nu = p->S;
  } else if (p->model == OR_PPLATE) {
    if (p->g < 4) return -1;  /* g = n grid points per side; the states are the (n-2)^2 interior nodes */
    p->nx = (p->g - 2) * (p->g - 2); p->nu = 1;
  } else if (p->model == OR_DDAE) {
    /* eq. (distill-ocp) with its algebraic variables: per stage [x (N) | y (N) u L V S],
     * per step N balances, N equilibria and the 3 flow equations */
    p->nx = p->N; p->nu = p->N + 4;
  } else { p->nx = 1; p->nu = 1; }
  if (p->T < 1) return -1;
  p->nr = (p->model == OR_DDAE) ? 2 * p->N + 3 : p->nx;
  p->n = p->nx + p->T * (p->nx + p->nu);
  p->m = p->nx + p->T * p->nr;
  return 0;
}

int or_jac_nnz(const or_problem* p) {
  int nnz = p->nx;
  for (int i = 0; i < p->nx; ++i) {
    int per;
    if (p->model == OR_DISTILL) per = 1 + (i > 0) + 1 + (i < p->nx - 1) + 1;
    else if (p->model == OR_PLATE) {
      const int g = p->g, ci = i % g, cj = i / g;
      int segs[2];
      per = 1 + 1 + (ci > 0) + (ci < g - 1) + (cj > 0) + (cj < g - 1) + or_plate_cell_segments(p, i, segs);
    } else if (p->model == OR_PPLATE) {
      const int mm = p->g - 2, ii = i % mm, jj = i / mm; /* interior node (ii + 1, jj + 1) */
      per = 1 + 1 + (ii > 0) + (ii < mm - 1) + (jj > 0) + (jj < mm - 1) + (ii == 0 || jj == 0);
    } else if (p->model == OR_DDAE) {
      per = 0; /* counted below by row kind */
    } else per = 3;
    nnz += per * p->T;
  }
  if (p->model == OR_DDAE) {
    const int N = p->N, Nf = p->Nf;
    int step = 0;
    for (int i = 1; i <= N; ++i) {
      /* x_k,i, the x_{k+1} neighbours, the y_{k+1} entries, the flows */
      if (i == 1) step += 1 + 1 + 1 + 1;                  /* x_k1 | x1 | y2 | V */
      else if (i == N) step += 1 + 2 + 1 + 2;             /* x_kN | x_{N-1} x_N | y_N | V S */
      else if (i < Nf) step += 1 + 2 + 2 + 2;             /* | x_{i-1} x_i | y_i y_{i+1} | L V */
      else if (i == Nf) step += 1 + 2 + 2 + 3;            /* | ... | L V S */
      else step += 1 + 2 + 2 + 2;                         /* | ... | V S */
    }
    step += 2 * N;      /* equilibria: x_i, y_i */
    step += 2 + 2 + 2;  /* L - u D, V - L - D, S - L - F */
    nnz += step * p->T;
  }
  return nnz;
}

/* variable bounds: x_0 is free (fixed by its equality); x_k, u_k for k >= 1
 * carry the model bounds */
void or_bounds(const or_problem* p, double* yL, double* yU) {
  for (int i = 0; i < p->nx; ++i) { yL[i] = -INFINITY; yU[i] = INFINITY; }
  for (int k = 1; k <= p->T; ++k) {
    int ox = or_off_x(p, k), ou = or_off_u(p, k);
    for (int i = 0; i < p->nx; ++i) { yL[ox + i] = p->xlo; yU[ox + i] = p->xhi; }
    for (int s = 0; s < p->nu; ++s) { yL[ou + s] = p->ulo; yU[ou + s] = p->uhi; }
    if (p->model == OR_DDAE) { /* y in [0, 1], u in [ulo, uhi], L, V, S in [0, 10] (eq. distill-ocp) */
      for (int s = 0; s < p->N; ++s) { yL[ou + s] = 0.0; yU[ou + s] = 1.0; }
      for (int s = p->N + 1; s < p->N + 4; ++s) { yL[ou + s] = 0.0; yU[ou + s] = 10.0; }
    }
  }
}

void or_eval(const or_problem* p, const double* y, double* f, double* grad, double* h,
             int* rowptr, int* colidx, double* Hvals) {
  if (f) *f = or_objective_d(p, y);
  if (grad) or_objective_grad_d(p, y, grad);
  if (h) or_constraints_d(p, y, h);
  if (Hvals) or_jacobian_d(p, y, rowptr, colidx, Hvals);
}

void or_eval_complex(const or_problem* p, const double* y_re, const double* y_im,
                     double* f_ri, double* grad_ri, double* h_ri, double* H_ri) {
  const int n = p->n, m = p->m, nnz = or_jac_nnz(p);
  double complex* y = malloc(sizeof(double complex) * n);
  double complex* g = malloc(sizeof(double complex) * n);
  double complex* h = malloc(sizeof(double complex) * m);
  double complex* H = malloc(sizeof(double complex) * nnz);
  int* rp = malloc(sizeof(int) * (m + 1));
  int* ci = malloc(sizeof(int) * nnz);
  for (int i = 0; i < n; ++i) y[i] = y_re[i] + I * y_im[i];
  double complex f = or_objective_z(p, y);
  or_objective_grad_z(p, y, g);
  or_constraints_z(p, y, h);
  or_jacobian_z(p, y, rp, ci, H);
  f_ri[0] = creal(f); f_ri[1] = cimag(f);
  for (int i = 0; i < n; ++i) { grad_ri[i] = creal(g[i]); grad_ri[n + i] = cimag(g[i]); }
  for (int i = 0; i < m; ++i) { h_ri[i] = creal(h[i]); h_ri[m + i] = cimag(h[i]); }
  for (int i = 0; i < nnz; ++i) { H_ri[i] = creal(H[i]); H_ri[nnz + i] = cimag(H[i]); }
  free(y); free(g); free(h); free(H); free(rp); free(ci);
}

/* ------------------------------------------------- Hessian of Lagrangian */

static int push_trip(int* rows, int* cols, double* vals, int cap, int k, int i, int j, double v) {
  if (k < cap) {
    if (i < j) { int t = i; i = j; j = t; }
    rows[k] = i; cols[k] = j; vals[k] = v;
  }
  return k + 1;
}

/* W = grad^2 f + sum_r lam_r grad^2 h_r as lower-triangle triplets (duplicates
 * allowed, to be summed).  Returns the number of triplets (may exceed cap). */
int or_hessian(const or_problem* p, const double* y, const double* lam,
               int* rows, int* cols, double* vals, int cap) {
  int k = 0;
  const int nx = p->nx;
  for (int t = 1; t <= p->T; ++t) {
    int ox = or_off_x(p, t), ou = or_off_u(p, t);
    if (p->model == OR_DISTILL || p->model == OR_DDAE) {
      const int cu = (p->model == OR_DDAE) ? p->N : 0;  /* u within the control block */
      k = push_trip(rows, cols, vals, cap, k, ox, ox, 2.0 * p->dt);
      k = push_trip(rows, cols, vals, cap, k, ou + cu, ou + cu, 2.0 * p->wdu + 2.0 * p->wu * p->dt);
      if (t > 1) {
        int oup = or_off_u(p, t - 1) + cu;
        k = push_trip(rows, cols, vals, cap, k, oup, oup, 2.0 * p->wdu);
        k = push_trip(rows, cols, vals, cap, k, ou + cu, oup, -2.0 * p->wdu);
      }
    } else if (p->model == OR_PLATE) {
      const double h = 1.0 / p->g;
      for (int c = 0; c < nx; ++c) k = push_trip(rows, cols, vals, cap, k, ox + c, ox + c, 2.0 * p->dt * h * h);
      for (int s = 0; s < p->nu; ++s) k = push_trip(rows, cols, vals, cap, k, ou + s, ou + s, 2.0 * p->rho_u * p->dt);
    } else if (p->model == OR_PPLATE) {
      for (int c = 0; c < nx; ++c) {
        const double w = pplate_weight_d(p, c);
        if (w != 0.0) k = push_trip(rows, cols, vals, cap, k, ox + c, ox + c, 2.0 * p->dt * w);
      }
      k = push_trip(rows, cols, vals, cap, k, ou, ou, 2.0 * p->rho_u * p->dt);
    } else {
      k = push_trip(rows, cols, vals, cap, k, ox, ox, 2.0 * p->dt);
    }
  }
  if (p->model == OR_PLATE) return k; /* linear dynamics */
  if (p->model == OR_DDAE) {
    /* the balances are bilinear in (flow, composition); the equilibria carry
     * -vle(x), whose second derivative is -2 a (a - 1) / (1 + (a - 1) x)^3 */
    const int N = p->N, Nf = p->Nf;
    const double a = p->alpha;
    for (int t = 0; t < p->T; ++t) {
      const int oxn = or_off_x(p, t + 1), oun = or_off_u(p, t + 1);
      const int cL = oun + N + 1, cV = oun + N + 2, cS = oun + N + 3;
      const double* lk = lam + nx + p->nr * t;
      for (int i = 1; i <= N; ++i) {
        const double c = -p->dt * lk[i - 1];  /* the balance carries -dt f_i */
        if (i == 1) {
          k = push_trip(rows, cols, vals, cap, k, cV, oun + 1, c / p->Ac);
          k = push_trip(rows, cols, vals, cap, k, cV, oxn, -c / p->Ac);
        } else if (i == N) {
          k = push_trip(rows, cols, vals, cap, k, cS, oxn + N - 2, c / p->Ar);
          k = push_trip(rows, cols, vals, cap, k, cV, oun + N - 1, -c / p->Ar);
        } else {
          const int cin = (i <= Nf) ? cL : cS, cout = (i < Nf) ? cL : cS;
          k = push_trip(rows, cols, vals, cap, k, cin, oxn + i - 2, c / p->At);
          k = push_trip(rows, cols, vals, cap, k, cout, oxn + i - 1, -c / p->At);
          k = push_trip(rows, cols, vals, cap, k, cV, oun + i - 1, -c / p->At);
          k = push_trip(rows, cols, vals, cap, k, cV, oun + i, c / p->At);
        }
      }
      for (int i = 0; i < N; ++i) {
        const double den = 1.0 + (a - 1.0) * y[oxn + i];
        k = push_trip(rows, cols, vals, cap, k, oxn + i, oxn + i, lk[N + i] * 2.0 * a * (a - 1.0) / (den * den * den));
      }
    }
    return k;
  }
  if (p->model == OR_PPLATE) {
    /* the dynamics are linear in T; the boundary data are not in Q:
     * d2/dQ2 4.1 Q^(1/3) = -(8.2/9) Q^(-5/3), d2/dQ2 Q^(1/2) = -Q^(-3/2) / 4 */
    const int n = p->g, mm = n - 2;
    const double h = 2.0 / (n - 1), c = p->kappa / (h * h), sc = pplate_row_scale_d(p);
    for (int t = 0; t < p->T; ++t) {
      const int oun = or_off_u(p, t + 1);
      const double Q = y[oun];
      const double* lk = lam + nx + p->nr * t;
      double s = 0.0;
      for (int q = 0; q < nx; ++q) {
        const int ii = q % mm + 1, jj = q / mm + 1;
        double d2 = 0.0;
        if (ii == 1) d2 += -(8.2 / 9.0) * pow(Q, -5.0 / 3.0);
        if (jj == 1) d2 += -0.25 * pow(Q, -1.5);
        s += lk[q] * sc * (-p->dt * c * d2);  /* the (scaled) constraint carries -sc dt f */
      }
      k = push_trip(rows, cols, vals, cap, k, oun, oun, s);
    }
    return k;
  }
  for (int t = 0; t < p->T; ++t) {
    const int oxn = or_off_x(p, t + 1), oun = or_off_u(p, t + 1);
    const double* xn = y + oxn;
    const double u = y[oun];
    const double* lk = lam + nx + p->nr * t;
    if (p->model == OR_TOY) {
      k = push_trip(rows, cols, vals, cap, k, oxn, oxn, lk[0] * 6.0 * p->dt * xn[0]);
      k = push_trip(rows, cols, vals, cap, k, oun, oun, lk[0] * 4.0 * p->dt * sin(u));
      continue;
    }
    const double a = p->alpha, D = p->D, V = (u + 1.0) * D;
    for (int i = 1; i <= nx; ++i) {
      /* second derivatives of f_i; the constraint carries -dt f_i */
      const double c = -p->dt * lk[i - 1];
      double yp[3], ypp[3]; /* y', y'' at x_{i-1}, x_i, x_{i+1} */
      for (int q = -1; q <= 1; ++q) {
        int idx = i - 1 + q;
        if (idx < 0 || idx >= nx) { yp[q + 1] = ypp[q + 1] = 0.0; continue; }
        double den = 1.0 + (a - 1.0) * xn[idx];
        yp[q + 1] = a / (den * den);
        ypp[q + 1] = -2.0 * a * (a - 1.0) / (den * den * den);
      }
      if (i == 1) {
        k = push_trip(rows, cols, vals, cap, k, oxn + 1, oxn + 1, c * V * ypp[2] / p->Ac);
        k = push_trip(rows, cols, vals, cap, k, oun, oxn + 0, c * (-D) / p->Ac);
        k = push_trip(rows, cols, vals, cap, k, oun, oxn + 1, c * D * yp[2] / p->Ac);
      } else if (i == nx) {
        k = push_trip(rows, cols, vals, cap, k, oxn + i - 1, oxn + i - 1, c * (-V * ypp[1]) / p->Ar);
        k = push_trip(rows, cols, vals, cap, k, oun, oxn + i - 2, c * D / p->Ar);
        k = push_trip(rows, cols, vals, cap, k, oun, oxn + i - 1, c * (-D * yp[1]) / p->Ar);
      } else {
        k = push_trip(rows, cols, vals, cap, k, oxn + i - 1, oxn + i - 1, c * (-V * ypp[1]) / p->At);
        k = push_trip(rows, cols, vals, cap, k, oxn + i, oxn + i, c * (V * ypp[2]) / p->At);
        k = push_trip(rows, cols, vals, cap, k, oun, oxn + i - 2, c * D / p->At);
        k = push_trip(rows, cols, vals, cap, k, oun, oxn + i - 1, c * (-D - D * yp[1]) / p->At);
        k = push_trip(rows, cols, vals, cap, k, oun, oxn + i, c * (D * yp[2]) / p->At);
      }
    }
  }
  return k;
}

/* ------------------------------------------------- distillation steady state */

/* Newton's method on f(x, u) = 0 (N unknowns, dense Gaussian elimination with
 * partial pivoting).  Returns the number of iterations, or -1. */
int or_steady_state(const or_problem* p, double u, double* x) {
  const int N = p->N;
  double* J = malloc(sizeof(double) * N * N);
  double* r = malloc(sizeof(double) * N);
  int it, ok = -1;
  for (int i = 0; i < N; ++i) x[i] = 0.5;
  for (it = 0; it < 100; ++it) {
    double rn = 0.0;
    for (int i = 1; i <= N; ++i) { r[i - 1] = distill_rhs_d(p, x, u, i); rn = fmax(rn, fabs(r[i - 1])); }
    if (rn < 1e-15) { ok = it; break; }
    memset(J, 0, sizeof(double) * N * N);
    for (int i = 1; i <= N; ++i) {
      double dm, d0, dp, du;
      distill_rhs_grad_d(p, x, u, i, &dm, &d0, &dp, &du);
      if (i > 1) J[(i - 1) * N + i - 2] = dm;
      J[(i - 1) * N + i - 1] = d0;
      if (i < N) J[(i - 1) * N + i] = dp;
    }
    /* solve J d = -r */
    for (int i = 0; i < N; ++i) r[i] = -r[i];
    for (int c = 0; c < N; ++c) {
      int piv = c;
      for (int q = c + 1; q < N; ++q) if (fabs(J[q * N + c]) > fabs(J[piv * N + c])) piv = q;
      if (piv != c) {
        for (int q = 0; q < N; ++q) { double t = J[c * N + q]; J[c * N + q] = J[piv * N + q]; J[piv * N + q] = t; }
        double t = r[c]; r[c] = r[piv]; r[piv] = t;
      }
      for (int q = c + 1; q < N; ++q) {
        double l = J[q * N + c] / J[c * N + c];
        for (int w = c; w < N; ++w) J[q * N + w] -= l * J[c * N + w];
        r[q] -= l * r[c];
      }
    }
    for (int c = N - 1; c >= 0; --c) {
      double s = r[c];
      for (int w = c + 1; w < N; ++w) s -= J[c * N + w] * r[w];
      r[c] = s / J[c * N + c];
    }
    for (int i = 0; i < N; ++i) x[i] += r[i];
  }
  free(J); free(r);
  return ok;
}

/* ------------------------------------------------------ banded Cholesky */

/* In-place Cholesky of a symmetric positive-definite band matrix.
 * band[j*(b+1) + d] holds K(j+d, j), d = 0..b (lower band, column-major).
 * eq. (cholesky-numeric): L_jj = sqrt(K_jj - sum L_js^2),
 * L_ij = (K_ij - sum L_is L_js) / L_jj.
 * Returns 0 on success, j+1 if the pivot of column j is not positive/finite. */
int or_band_cholesky(int n, int b, double* band) {
  const int w = b + 1;
  for (int j = 0; j < n; ++j) {
    double* cj = band + (size_t)j * w;
    double d = cj[0];
    if (!(d > 0.0) || !isfinite(d)) return j + 1;
    d = sqrt(d);
    cj[0] = d;
    const int len = (n - 1 - j < b) ? n - 1 - j : b;
    for (int i = 1; i <= len; ++i) cj[i] /= d;
    /* right-looking update of the trailing band */
    for (int q = 1; q <= len; ++q) {
      double* cq = band + (size_t)(j + q) * w;
      const double l = cj[q];
      for (int i = q; i <= len; ++i) cq[i - q] -= cj[i] * l;
    }
  }
  return 0;
}

/* Cholesky with a relative pivot tolerance: column j's pivot must exceed
 * tol * |K_jj| (K_jj the diagonal entry before factorization).  With tol > 0 a
 * pivot at rounding level counts as a zero eigenvalue, i.e. the wrong inertia
 * of eq. (infiniteOCP-inertia), which requires n_0 = 0. */
static int band_cholesky_tol(int n, int b, double* band, double tol) {
  const int w = b + 1;
  if (tol <= 0.0) return or_band_cholesky(n, b, band);
  double* diag = malloc(sizeof(double) * n);
  for (int j = 0; j < n; ++j) diag[j] = fabs(band[(size_t)j * w]);
  int rc = 0;
  for (int j = 0; j < n && rc == 0; ++j) {
    double* cj = band + (size_t)j * w;
    double d = cj[0];
    if (!(d > tol * diag[j]) || !(d > 0.0) || !isfinite(d)) { rc = j + 1; break; }
    d = sqrt(d);
    cj[0] = d;
    const int len = (n - 1 - j < b) ? n - 1 - j : b;
    for (int i = 1; i <= len; ++i) cj[i] /= d;
    for (int q = 1; q <= len; ++q) {
      double* cq = band + (size_t)(j + q) * w;
      const double l = cj[q];
      for (int i = q; i <= len; ++i) cq[i - q] -= cj[i] * l;
    }
  }
  free(diag);
  return rc;
}

static void band_solve(int n, int b, const double* band, double* x) {
  const int w = b + 1;
  for (int j = 0; j < n; ++j) {           /* L v = x */
    const double* cj = band + (size_t)j * w;
    x[j] /= cj[0];
    const int len = (n - 1 - j < b) ? n - 1 - j : b;
    for (int i = 1; i <= len; ++i) x[j + i] -= cj[i] * x[j];
  }
  for (int j = n - 1; j >= 0; --j) {      /* L^T x = v */
    const double* cj = band + (size_t)j * w;
    const int len = (n - 1 - j < b) ? n - 1 - j : b;
    double s = x[j];
    for (int i = 1; i <= len; ++i) s -= cj[i] * x[j + i];
    x[j] = s / cj[0];
  }
}

/* ------------------------------------------------------ SymCholesky */

static int cmp_int(const void* a, const void* b) {
  const int x = *(const int*)a, y = *(const int*)b;
  return (x > y) - (x < y);
}

/* Symbolic factorization as described in Sec. 3.2.3: the parent of column j
 * in the elimination tree is the first off-diagonal row of column j of L, and
 * the structure of column j of L is the structure of column j of the (lower)
 * matrix united with the structures of its children, without the child's own
 * row.  Columns are processed in increasing order so children come first; each
 * column joins its parent's list of children once its structure is known.
 * Input: lower-triangular pattern in CSC (diagonal optional, rows sorted or
 * not).  Output: parent (-1 = root) and the pattern of L as malloc'd CSC
 * arrays (rows sorted, diagonal included).  Returns nnz(L), or -1 if out of
 * memory or above the int range. */
static long symbolic_alloc(int n, const int* colptr, const int* rowidx, int* parent,
                           int** Lcolptr, int** Lrowidx) {
  const int nn = n > 0 ? n : 1;
  int* mark = malloc(sizeof(int) * nn);
  int* child = malloc(sizeof(int) * nn);  /* first child of each column */
  int* sib = malloc(sizeof(int) * nn);    /* next child of the same parent */
  int** cols = calloc(nn, sizeof(int*));
  int* cnt = calloc(nn, sizeof(int));
  int* buf = malloc(sizeof(int) * nn);
  long total = 0;
  int ok = mark && child && sib && cols && cnt && buf;
  for (int j = 0; ok && j < n; ++j) { mark[j] = -1; child[j] = -1; }
  for (int j = 0; ok && j < n; ++j) {
    int k = 0;
    buf[k++] = j;
    mark[j] = j;
    for (int e = colptr[j]; e < colptr[j + 1]; ++e) {
      const int i = rowidx[e];
      if (i > j && mark[i] != j) { mark[i] = j; buf[k++] = i; }
    }
    for (int c = child[j]; c >= 0; c = sib[c])
      for (int q = 0; q < cnt[c]; ++q) {
        const int i = cols[c][q];
        if (i > j && mark[i] != j) { mark[i] = j; buf[k++] = i; }
      }
    qsort(buf, k, sizeof(int), cmp_int);
    cols[j] = malloc(sizeof(int) * k);
    if (!cols[j]) { ok = 0; break; }
    memcpy(cols[j], buf, sizeof(int) * k);
    cnt[j] = k;
    parent[j] = k > 1 ? buf[1] : -1;
    if (k > 1) { sib[j] = child[buf[1]]; child[buf[1]] = j; }
    total += k;
  }
  if (total > 2147483647L) ok = 0;
  if (ok) {
    *Lcolptr = malloc(sizeof(int) * (nn + 1));
    *Lrowidx = malloc(sizeof(int) * (total > 0 ? total : 1));
    ok = *Lcolptr && *Lrowidx;
  }
  if (ok) {
    int e = 0;
    for (int j = 0; j < n; ++j) {
      (*Lcolptr)[j] = e;
      memcpy(*Lrowidx + e, cols[j], sizeof(int) * cnt[j]);
      e += cnt[j];
    }
    (*Lcolptr)[n] = e;
  }
  for (int j = 0; cols && j < n; ++j) free(cols[j]);
  free(cols); free(cnt); free(mark); free(child); free(sib); free(buf);
  return ok ? total : -1;
}

/* or_symbolic: the same into caller arrays; returns nnz(L), or -1 if cap is
 * too small. */
int or_symbolic(int n, const int* colptr, const int* rowidx, int* parent,
                int* Lcolptr, int* Lrowidx, int cap) {
  int *Lp = NULL, *Li = NULL;
  const long total = symbolic_alloc(n, colptr, rowidx, parent, &Lp, &Li);
  if (total < 0 || total > cap) { free(Lp); free(Li); return -1; }
  memcpy(Lcolptr, Lp, sizeof(int) * (n + 1));
  memcpy(Lrowidx, Li, sizeof(int) * total);
  free(Lp); free(Li);
  return (int)total;
}

#include "or_sparse.inc"

/* ------------------------------------------------------ interior point */

/* Constants of the interior-point method (Wachter & Biegler 2006 defaults). */
#define KAPPA_EPS 10.0      /* barrier subproblem tolerance factor */
#define KAPPA_MU 0.2        /* linear barrier decrease */
#define THETA_MU 1.5        /* superlinear barrier decrease */
#define TAU_MIN 0.99        /* fraction-to-the-boundary */
#define S_MAX 100.0         /* scaling threshold of the optimality error */
#define KAPPA_SIGMA 1e10    /* bound-multiplier safeguard */
#define GAMMA_THETA 1e-5
#define GAMMA_PHI 1e-5
#define DELTA_SW 1.0
#define S_THETA 1.1
#define S_PHI 2.3
#define ETA_PHI 1e-4
#define GAMMA_ALPHA 0.05
#define DELTA_W0 1e-4       /* first regularization trial */
#define DELTA_WMIN 1e-20
#define KAPPA_W_MINUS (1.0 / 3.0)
#define KAPPA_W_PLUS 8.0
#define KAPPA_W_PLUS_BAR 100.0

typedef struct {
  const or_problem* p;
  const or_options* o;
  int n, m, nnz, b, ntrip_cap;
  double *yL, *yU;
  double f, *grad, *h, *Hv;
  int *rp, *ci;
  int *tr, *tc; double *tv; /* Hessian triplets */
  double *band, *rhs, *lam, *tmp;
  double *gv, *cg_r, *cg_p, *cg_q, *cg_x; /* HyKKT: right-hand side g (n), CG vectors (m) */
  int nL, nU;
  int sparse;      /* options.linsolve = 1: K in the sparse factor below, band unused */
  sp_factor spf;
} work;

static int cmp_long(const void* a, const void* b) {
  const long x = *(const long*)a, y = *(const long*)b;
  return (x > y) - (x < y);
}

/* Lower pattern of K = W + Sigma_y + delta_w I + H^T D H as CSC without
 * duplicates: the Hessian triplets, the diagonal and every pair of columns
 * of one Jacobian row.  Sets up the sparse factor on it. */
static int sparse_init(work* w, int cnt) {
  const int n = w->n, m = w->m;
  long np = (long)cnt + n;
  for (int r = 0; r < m; ++r) { const long k = w->rp[r + 1] - w->rp[r]; np += k * (k + 1) / 2; }
  long* key = malloc(sizeof(long) * np);
  if (!key) return -1;
  long q = 0;
  for (int t = 0; t < cnt; ++t) key[q++] = (long)w->tc[t] * n + w->tr[t];
  for (int i = 0; i < n; ++i) key[q++] = (long)i * n + i;
  for (int r = 0; r < m; ++r)
    for (int a = w->rp[r]; a < w->rp[r + 1]; ++a)
      for (int c = w->rp[r]; c <= a; ++c) key[q++] = (long)w->ci[c] * n + w->ci[a];
  qsort(key, np, sizeof(long), cmp_long);
  int* colptr = calloc(n + 1, sizeof(int));
  int* rowidx = malloc(sizeof(int) * np);
  long u = 0;
  for (long e = 0; e < np; ++e) {
    if (e > 0 && key[e] == key[e - 1]) continue;
    ++colptr[key[e] / n + 1];
    rowidx[u++] = (int)(key[e] % n);
  }
  for (int j = 0; j < n; ++j) colptr[j + 1] += colptr[j];
  free(key);
  const int rc = sp_setup(&w->spf, n, colptr, rowidx, 1);
  free(colptr); free(rowidx);
  return rc;
}

/* add v to K(i, j), i >= j */
static inline void kadd(work* w, int i, int j, double v) {
  if (w->sparse) sp_add(&w->spf, i, j, v);
  else w->band[(size_t)j * (w->b + 1) + (i - j)] += v;
}

/* factor K in place with the inertia test's pivot tolerance; 0 on success */
static int kfactor(work* w, double tol) {
  return w->sparse ? sp_cholesky_tol(&w->spf, tol) : band_cholesky_tol(w->n, w->b, w->band, tol);
}

/* x <- K^-1 x with the factor of kfactor */
static void ksolve(work* w, double* x) {
  if (w->sparse) sp_solve(&w->spf, x);
  else band_solve(w->n, w->b, w->band, x);
}

static int work_init(work* w, const or_problem* p, const or_options* o) {
  memset(w, 0, sizeof(*w));
  w->p = p; w->o = o;
  w->n = p->n; w->m = p->m; w->nnz = or_jac_nnz(p);
  const int n = w->n, m = w->m;
  w->yL = malloc(sizeof(double) * n); w->yU = malloc(sizeof(double) * n);
  or_bounds(p, w->yL, w->yU);
  w->nL = w->nU = 0;
  for (int i = 0; i < n; ++i) { w->nL += isfinite(w->yL[i]); w->nU += isfinite(w->yU[i]); }
  w->grad = malloc(sizeof(double) * n); w->h = malloc(sizeof(double) * m);
  w->Hv = malloc(sizeof(double) * w->nnz);
  w->rp = malloc(sizeof(int) * (m + 1)); w->ci = malloc(sizeof(int) * w->nnz);
  w->lam = calloc(m, sizeof(double));
  double* y0 = calloc(n, sizeof(double));
  int cnt = or_hessian(p, y0, w->lam, NULL, NULL, NULL, 0);
  w->ntrip_cap = cnt;
  w->tr = malloc(sizeof(int) * cnt); w->tc = malloc(sizeof(int) * cnt); w->tv = malloc(sizeof(double) * cnt);
  or_hessian(p, y0, w->lam, w->tr, w->tc, w->tv, cnt);
  /* bandwidth from the Jacobian rows and Hessian triplets */
  or_eval(p, y0, NULL, NULL, NULL, w->rp, w->ci, w->Hv);
  int b = 0;
  for (int r = 0; r < m; ++r) {
    int lo = w->ci[w->rp[r]], hi = w->ci[w->rp[r + 1] - 1];
    if (hi - lo > b) b = hi - lo;
  }
  for (int t = 0; t < cnt; ++t) if (w->tr[t] - w->tc[t] > b) b = w->tr[t] - w->tc[t];
  w->b = b;
  free(y0);
  w->sparse = o->linsolve == 1;
  if (w->sparse) { if (sparse_init(w, cnt) != 0) return -1; }
  else w->band = malloc(sizeof(double) * (size_t)(b + 1) * n);
  w->rhs = malloc(sizeof(double) * n);
  w->tmp = malloc(sizeof(double) * (n > m ? n : m));
  w->gv = malloc(sizeof(double) * n);
  w->cg_r = malloc(sizeof(double) * m); w->cg_p = malloc(sizeof(double) * m);
  w->cg_q = malloc(sizeof(double) * m); w->cg_x = malloc(sizeof(double) * m);
  return ((w->band || w->sparse) && w->rhs && w->gv && w->cg_r && w->cg_p && w->cg_q && w->cg_x) ? 0 : -1;
}

static void work_free(work* w) {
  free(w->yL); free(w->yU); free(w->grad); free(w->h); free(w->Hv); free(w->rp); free(w->ci);
  free(w->lam); free(w->tr); free(w->tc); free(w->tv); free(w->band); free(w->rhs); free(w->tmp);
  free(w->gv); free(w->cg_r); free(w->cg_p); free(w->cg_q); free(w->cg_x);
  if (w->sparse) sp_free(&w->spf);
}

static void eval_all(work* w, const double* y) {
  or_eval(w->p, y, &w->f, w->grad, w->h, w->rp, w->ci, w->Hv);
}

/* H^T v (length n) */
static void jac_t_mult(const work* w, const double* v, double* out) {
  for (int i = 0; i < w->n; ++i) out[i] = 0.0;
  for (int r = 0; r < w->m; ++r)
    for (int e = w->rp[r]; e < w->rp[r + 1]; ++e) out[w->ci[e]] += w->Hv[e] * v[r];
}

/* H v (length m) */
static void jac_mult(const work* w, const double* v, double* out) {
  for (int r = 0; r < w->m; ++r) {
    double s = 0.0;
    for (int e = w->rp[r]; e < w->rp[r + 1]; ++e) s += w->Hv[e] * v[w->ci[e]];
    out[r] = s;
  }
}

/* Optimality error E_mu of the lifted barrier problem (W&B eq. (5)):
 * stationarity in y and s scaled by s_d, constraint violation, and
 * complementarity scaled by s_c.  Uses w->grad, w->h, w->Hv at z->y. */
static void errors(work* w, const or_state* z, double mu, double* Es, double* Eu) {
  const int n = w->n, m = w->m;
  const double gam = w->o->gamma;
  double* ry = w->tmp;
  for (int r = 0; r < m; ++r) w->lam[r] = z->w_p[r] - z->w_m[r];
  jac_t_mult(w, w->lam, ry);
  double dual = 0.0, prim = 0.0, comp = 0.0, sum_l = 0.0, sum_z = 0.0;
  for (int i = 0; i < n; ++i) {
    double v = w->grad[i] + ry[i];
    if (isfinite(w->yL[i])) { v -= z->zL[i]; sum_z += fabs(z->zL[i]); comp = fmax(comp, fabs((z->y[i] - w->yL[i]) * z->zL[i] - mu)); }
    if (isfinite(w->yU[i])) { v += z->zU[i]; sum_z += fabs(z->zU[i]); comp = fmax(comp, fabs((w->yU[i] - z->y[i]) * z->zU[i] - mu)); }
    dual = fmax(dual, fabs(v));
  }
  for (int r = 0; r < m; ++r) {
    dual = fmax(dual, fabs(z->w_p[r] - z->b_p[r]));
    dual = fmax(dual, fabs(z->w_m[r] - z->b_m[r]));
    prim = fmax(prim, fabs(w->h[r] - gam + z->s_p[r]));
    prim = fmax(prim, fabs(-w->h[r] - gam + z->s_m[r]));
    comp = fmax(comp, fabs(z->s_p[r] * z->b_p[r] - mu));
    comp = fmax(comp, fabs(z->s_m[r] * z->b_m[r] - mu));
    sum_l += fabs(z->w_p[r]) + fabs(z->w_m[r]);
    sum_z += fabs(z->b_p[r]) + fabs(z->b_m[r]);
  }
  const double nz = (double)(w->nL + w->nU + 2 * m);
  const double sd = fmax(S_MAX, (sum_l + sum_z) / (2.0 * m + nz)) / S_MAX;
  const double sc = fmax(S_MAX, sum_z / nz) / S_MAX;
  *Es = fmax(fmax(dual / sd, prim), comp / sc);
  if (Eu) *Eu = fmax(fmax(dual, prim), comp);
}

/* Optimality error E_mu of the barrier problem with its equalities kept
 * (HyKKT form, W&B eq. (5) as printed there): stationarity
 * grad f + H^T lambda - zL + zU scaled by s_d, the constraint values h, and
 * the bound complementarity scaled by s_c; s_d averages |lambda| and z over
 * the m + n_z multipliers, s_c averages z over the n_z bound multipliers. */
static void errors_hy(work* w, const or_state* z, double mu, double* Es, double* Eu) {
  const int n = w->n, m = w->m;
  double* ry = w->tmp;
  jac_t_mult(w, z->w_p, ry);
  double dual = 0.0, prim = 0.0, comp = 0.0, sum_l = 0.0, sum_z = 0.0;
  for (int i = 0; i < n; ++i) {
    double v = w->grad[i] + ry[i];
    if (isfinite(w->yL[i])) { v -= z->zL[i]; sum_z += fabs(z->zL[i]); comp = fmax(comp, fabs((z->y[i] - w->yL[i]) * z->zL[i] - mu)); }
    if (isfinite(w->yU[i])) { v += z->zU[i]; sum_z += fabs(z->zU[i]); comp = fmax(comp, fabs((w->yU[i] - z->y[i]) * z->zU[i] - mu)); }
    dual = fmax(dual, fabs(v));
  }
  for (int r = 0; r < m; ++r) {
    prim = fmax(prim, fabs(w->h[r]));
    sum_l += fabs(z->w_p[r]);
  }
  const double nz = (double)(w->nL + w->nU);
  const double sd = fmax(S_MAX, (sum_l + sum_z) / (m + nz)) / S_MAX;
  const double sc = fmax(S_MAX, sum_z / nz) / S_MAX;
  *Es = fmax(fmax(dual / sd, prim), comp / sc);
  if (Eu) *Eu = fmax(fmax(dual, prim), comp);
}

/* barrier objective phi_mu and constraint violation theta (1-norm) of the
 * HyKKT form: phi = f - mu sum log(bound gaps), theta = ||h||_1 */
static void merit_hy(work* w, const double* y, double f, const double* h, double mu,
                     double* phi, double* theta) {
  double lg = 0.0, th = 0.0;
  for (int i = 0; i < w->n; ++i) {
    if (isfinite(w->yL[i])) lg += log(y[i] - w->yL[i]);
    if (isfinite(w->yU[i])) lg += log(w->yU[i] - y[i]);
  }
  for (int r = 0; r < w->m; ++r) th += fabs(h[r]);
  *phi = f - mu * lg;
  *theta = th;
}

/* barrier objective phi_mu and constraint violation theta (1-norm) at (y, s) */
static void merit(work* w, const double* y, const double* sp, const double* sm,
                  double f, const double* h, double mu, double* phi, double* theta) {
  const double gam = w->o->gamma;
  double lg = 0.0, th = 0.0;
  for (int i = 0; i < w->n; ++i) {
    if (isfinite(w->yL[i])) lg += log(y[i] - w->yL[i]);
    if (isfinite(w->yU[i])) lg += log(w->yU[i] - y[i]);
  }
  for (int r = 0; r < w->m; ++r) {
    lg += log(sp[r]) + log(sm[r]);
    th += fabs(h[r] - gam + sp[r]) + fabs(-h[r] - gam + sm[r]);
  }
  *phi = f - mu * lg;
  *theta = th;
}

/* the optimality error and the merits of the form the options select */
static void opt_error(work* w, const or_state* z, double mu, double* Es, double* Eu) {
  if (w->o->kkt == 1) errors_hy(w, z, mu, Es, Eu);
  else errors(w, z, mu, Es, Eu);
}
static void merit_of(work* w, const double* y, const double* sp, const double* sm,
                     double f, const double* h, double mu, double* phi, double* theta) {
  if (w->o->kkt == 1) merit_hy(w, y, f, h, mu, phi, theta);
  else merit(w, y, sp, sm, f, h, mu, phi, theta);
}

/* Assemble K_c = W + Sigma_y + delta_w I + H^T (Q+ + Q-) H into band or
 * sparse storage (eq. liftedkkt-pd), from w->grad/h/Hv evaluated at z->y.  In the HyKKT form
 * the same pattern holds K_gamma = W + Sigma_y + delta_w I + gamma H^T H, the
 * augmented-Lagrangian matrix, with W the Hessian at the multipliers lambda. */
static void assemble(work* w, const or_state* z, double delta_w) {
  const int n = w->n, m = w->m;
  const int hy = w->o->kkt == 1;
  if (w->sparse) memset(w->spf.Lx, 0, sizeof(double) * (size_t)w->spf.Lp[n]);
  else memset(w->band, 0, sizeof(double) * (size_t)(w->b + 1) * n);
  for (int r = 0; r < m; ++r) w->lam[r] = hy ? z->w_p[r] : z->w_p[r] - z->w_m[r];
  int cnt = or_hessian(w->p, z->y, w->lam, w->tr, w->tc, w->tv, w->ntrip_cap);
  for (int t = 0; t < cnt; ++t) kadd(w, w->tr[t], w->tc[t], w->tv[t]);
  for (int i = 0; i < n; ++i) {
    double sig = delta_w;
    if (isfinite(w->yL[i])) sig += z->zL[i] / (z->y[i] - w->yL[i]);
    if (isfinite(w->yU[i])) sig += z->zU[i] / (w->yU[i] - z->y[i]);
    kadd(w, i, i, sig);
  }
  for (int r = 0; r < m; ++r) {
    const double D = hy ? w->o->hy_gamma : z->b_p[r] / z->s_p[r] + z->b_m[r] / z->s_m[r];
    for (int a = w->rp[r]; a < w->rp[r + 1]; ++a)
      for (int c = w->rp[r]; c <= a; ++c) {
        const int i = w->ci[a], j = w->ci[c]; /* columns ascending: i >= j */
        kadd(w, i, j, D * w->Hv[a] * w->Hv[c]);
      }
  }
}

/* Newton direction from the factored K (eqs. liftedkkt-pd, cholesky-lower/
 * upper/delta and the eliminated rows of eq. infiniteOCP-augmented). */
static void direction(work* w, const or_state* z, double mu, or_state* d) {
  const int n = w->n, m = w->m;
  const double gam = w->o->gamma;
  /* r1 = grad f + H^T (w+ - w-) - mu/(y - yL) + mu/(yU - y)
   * rhs = -r1 - H^T [(Q+ r4+ - r2+) - (Q- r4- - r2-)] */
  double* v = w->tmp;
  for (int r = 0; r < m; ++r) {
    const double r4p = w->h[r] - gam + z->s_p[r], r4m = -w->h[r] - gam + z->s_m[r];
    const double r2p = z->w_p[r] - mu / z->s_p[r], r2m = z->w_m[r] - mu / z->s_m[r];
    const double Qp = z->b_p[r] / z->s_p[r], Qm = z->b_m[r] / z->s_m[r];
    v[r] = (z->w_p[r] - z->w_m[r]) + (Qp * r4p - r2p) - (Qm * r4m - r2m);
  }
  jac_t_mult(w, v, w->rhs);
  for (int i = 0; i < n; ++i) {
    double r1 = w->grad[i] + w->rhs[i];
    if (isfinite(w->yL[i])) r1 -= mu / (z->y[i] - w->yL[i]);
    if (isfinite(w->yU[i])) r1 += mu / (w->yU[i] - z->y[i]);
    w->rhs[i] = -r1;
  }
  memcpy(d->y, w->rhs, sizeof(double) * n);
  ksolve(w, d->y);
  /* recover the eliminated directions */
  double* Hd = w->tmp;
  jac_mult(w, d->y, Hd);
  for (int r = 0; r < m; ++r) {
    const double r4p = w->h[r] - gam + z->s_p[r], r4m = -w->h[r] - gam + z->s_m[r];
    const double Qp = z->b_p[r] / z->s_p[r], Qm = z->b_m[r] / z->s_m[r];
    d->s_p[r] = -r4p - Hd[r];
    d->s_m[r] = -r4m + Hd[r];
    d->w_p[r] = -(z->w_p[r] - mu / z->s_p[r]) - Qp * d->s_p[r];
    d->w_m[r] = -(z->w_m[r] - mu / z->s_m[r]) - Qm * d->s_m[r];
    d->b_p[r] = mu / z->s_p[r] - z->b_p[r] - Qp * d->s_p[r];
    d->b_m[r] = mu / z->s_m[r] - z->b_m[r] - Qm * d->s_m[r];
  }
  for (int i = 0; i < n; ++i) {
    d->zL[i] = d->zU[i] = 0.0;
    if (isfinite(w->yL[i])) {
      const double gap = z->y[i] - w->yL[i];
      d->zL[i] = mu / gap - z->zL[i] - z->zL[i] / gap * d->y[i];
    }
    if (isfinite(w->yU[i])) {
      const double gap = w->yU[i] - z->y[i];
      d->zU[i] = mu / gap - z->zU[i] + z->zU[i] / gap * d->y[i];
    }
  }
}

/* Newton direction of the HyKKT form from the factored K_gamma.  The
 * primal-dual system of the barrier problem with its equalities kept,
 *   [Wh  H^T] [dy  ]   [a]   a = -(grad phi_mu + H^T lambda)
 *   [H   0  ] [dlam] = [c],  c = -h,   Wh = W + Sigma_y + delta_w I,
 * is solved as in the hybrid direct-iterative method the paper cites
 * (Regev et al. 2023, after Golub & Greif 2003): adding gamma H^T times the
 * second block row to the first gives K_gamma dy + H^T dlam = a + gamma H^T c
 * =: g, so with S = H K_gamma^-1 H^T
 *   S dlam = H K_gamma^-1 g - c            (conjugate gradients on S),
 *   dy = K_gamma^-1 (g - H^T dlam)         (one more solve).
 * CG starts from dlam = 0 and stops when ||r||^2 <= cg_tol^2 ||r_0||^2, after
 * cg_max_iter iterations, or when p^T S p is not positive.  The bound
 * multipliers follow as in the lifted form.  Returns the CG iterations. */
static int direction_hy(work* w, const or_state* z, double mu, or_state* d) {
  const int n = w->n, m = w->m;
  const double gam = w->o->hy_gamma;
  double *g = w->gv, *r = w->cg_r, *p = w->cg_p, *q = w->cg_q, *x = w->cg_x, *v = w->rhs;
  /* g = -(grad phi_mu + H^T (lambda + gamma h)) */
  for (int i = 0; i < m; ++i) w->tmp[i] = z->w_p[i] + gam * w->h[i];
  jac_t_mult(w, w->tmp, g);
  for (int i = 0; i < n; ++i) {
    double gp = w->grad[i] + g[i];
    if (isfinite(w->yL[i])) gp -= mu / (z->y[i] - w->yL[i]);
    if (isfinite(w->yU[i])) gp += mu / (w->yU[i] - z->y[i]);
    g[i] = -gp;
  }
  /* r_0 = H K^-1 g - c = H K^-1 g + h */
  memcpy(v, g, sizeof(double) * n);
  ksolve(w, v);
  jac_mult(w, v, r);
  double rr = 0.0;
  for (int i = 0; i < m; ++i) { r[i] += w->h[i]; x[i] = 0.0; p[i] = r[i]; rr += r[i] * r[i]; }
  const double stop = w->o->cg_tol * w->o->cg_tol * rr;
  int it = 0;
  while (rr > stop && it < w->o->cg_max_iter) {
    /* q = S p = H K^-1 H^T p */
    jac_t_mult(w, p, v);
    ksolve(w, v);
    jac_mult(w, v, q);
    double pq = 0.0;
    for (int i = 0; i < m; ++i) pq += p[i] * q[i];
    if (!(pq > 0.0)) break;
    const double a = rr / pq;
    double rr_new = 0.0;
    for (int i = 0; i < m; ++i) { x[i] += a * p[i]; r[i] -= a * q[i]; rr_new += r[i] * r[i]; }
    const double beta = rr_new / rr;
    rr = rr_new;
    for (int i = 0; i < m; ++i) p[i] = r[i] + beta * p[i];
    ++it;
  }
  /* dy = K^-1 (g - H^T dlam) */
  jac_t_mult(w, x, v);
  for (int i = 0; i < n; ++i) d->y[i] = g[i] - v[i];
  ksolve(w, d->y);
  memcpy(d->w_p, x, sizeof(double) * m);
  for (int i = 0; i < n; ++i) {
    d->zL[i] = d->zU[i] = 0.0;
    if (isfinite(w->yL[i])) {
      const double gap = z->y[i] - w->yL[i];
      d->zL[i] = mu / gap - z->zL[i] - z->zL[i] / gap * d->y[i];
    }
    if (isfinite(w->yU[i])) {
      const double gap = w->yU[i] - z->y[i];
      d->zU[i] = mu / gap - z->zU[i] + z->zU[i] / gap * d->y[i];
    }
  }
  return it;
}

/* Inertia correction (W&B Algorithm IC restricted to delta_w, since the
 * lifted system has no equality block): factor with 0, then 1e-4 or
 * last/3, then x100 (first) or x8, failing above dw_max (1e40 by default).  Returns 0 on
 * success and sets *dw; -1 on failure. */
static int factor_with_correction(work* w, const or_state* z, double* dw_last, double* dw, int* retries) {
  const double tol = w->o->pivtol;
  assemble(w, z, 0.0);
  if (kfactor(w, tol) == 0) { *dw = 0.0; return 0; }
  double d = (*dw_last == 0.0) ? DELTA_W0 : fmax(DELTA_WMIN, KAPPA_W_MINUS * *dw_last);
  for (;;) {
    ++*retries;
    assemble(w, z, d);
    if (kfactor(w, tol) == 0) { *dw = d; *dw_last = d; return 0; }
    d = (*dw_last == 0.0) ? KAPPA_W_PLUS_BAR * d : KAPPA_W_PLUS * d;
    if (d > w->o->dw_max) return -1;
  }
}

static double frac_to_boundary(const double* v, const double* dv, double tau, int len, double amax) {
  for (int i = 0; i < len; ++i)
    if (dv[i] < 0.0) { double a = -tau * v[i] / dv[i]; if (a < amax) amax = a; }
  return amax;
}

/* push x into [lo, hi] as in W&B Sec. 3.6 with kappa_1 = kappa_2 = k */
static double push_into(double x, double lo, double hi, double k) {
  double pl = isfinite(lo) ? k * fmax(1.0, fabs(lo)) : 0.0;
  double pu = isfinite(hi) ? k * fmax(1.0, fabs(hi)) : 0.0;
  if (isfinite(lo) && isfinite(hi)) { pl = fmin(pl, k * (hi - lo)); pu = fmin(pu, k * (hi - lo)); }
  if (isfinite(lo) && x < lo + pl) x = lo + pl;
  if (isfinite(hi) && x > hi - pu) x = hi - pu;
  return x;
}

static int all_finite(const double* v, int len) {
  for (int i = 0; i < len; ++i) if (!isfinite(v[i])) return 0;
  return 1;
}

int or_solve(const or_problem* p, const or_options* o, or_state* z, int warm,
             or_info* info, double* trace, int trace_cap) {
  work w;
  memset(info, 0, sizeof(*info));
  if (work_init(&w, p, o)) { work_free(&w); info->status = 2; return 2; }
  const int n = w.n, m = w.m;
  const double gam = o->gamma;
  const int hy = o->kkt == 1;
  const double mu_min = o->tol / 10.0;
  double mu = warm ? o->mu0_warm : o->mu0_cold;
  const double push = warm ? o->push_warm : o->push_cold;

  /* initial point (Sec. 3.2.4: warm start from the previous solution) */
  for (int i = 0; i < n; ++i) z->y[i] = push_into(z->y[i], w.yL[i], w.yU[i], push);
  eval_all(&w, z->y);
  if (!warm && hy) {
    /* HyKKT form: equality multipliers start at 0 */
    for (int r = 0; r < m; ++r) z->w_p[r] = 0.0;
    for (int i = 0; i < n; ++i) {
      z->zL[i] = isfinite(w.yL[i]) ? 1.0 : 0.0;
      z->zU[i] = isfinite(w.yU[i]) ? 1.0 : 0.0;
    }
  } else if (!warm) {
    for (int r = 0; r < m; ++r) {
      z->s_p[r] = fmax(gam - w.h[r], push);
      z->s_m[r] = fmax(gam + w.h[r], push);
      z->w_p[r] = z->w_m[r] = 1.0;
      z->b_p[r] = z->b_m[r] = 1.0;
    }
    for (int i = 0; i < n; ++i) {
      z->zL[i] = isfinite(w.yL[i]) ? 1.0 : 0.0;
      z->zU[i] = isfinite(w.yU[i]) ? 1.0 : 0.0;
    }
  } else {
    for (int r = 0; r < m && !hy; ++r) {
      z->s_p[r] = fmax(z->s_p[r], push); z->s_m[r] = fmax(z->s_m[r], push);
      z->b_p[r] = fmax(z->b_p[r], push); z->b_m[r] = fmax(z->b_m[r], push);
    }
    for (int i = 0; i < n; ++i) {
      z->zL[i] = isfinite(w.yL[i]) ? fmax(z->zL[i], push) : 0.0;
      z->zU[i] = isfinite(w.yU[i]) ? fmax(z->zU[i], push) : 0.0;
    }
  }

  or_state d, zt;
  double* dbuf = malloc(sizeof(double) * (3 * n + 6 * m) * 2);
  d.y = dbuf; d.zL = d.y + n; d.zU = d.zL + n;
  d.s_p = d.zU + n; d.s_m = d.s_p + m; d.w_p = d.s_m + m; d.w_m = d.w_p + m; d.b_p = d.w_m + m; d.b_m = d.b_p + m;
  zt.y = d.b_m + m; zt.zL = zt.y + n; zt.zU = zt.zL + n;
  zt.s_p = zt.zU + n; zt.s_m = zt.s_p + m; zt.w_p = zt.s_m + m; zt.w_m = zt.w_p + m; zt.b_p = zt.w_m + m; zt.b_m = zt.b_p + m;
  double* ht = malloc(sizeof(double) * m);
  const int fcap = o->max_iter + 8;
  double* filt_th = malloc(sizeof(double) * fcap);
  double* filt_ph = malloc(sizeof(double) * fcap);
  int nf = 0;

  double phi, theta;
  merit_of(&w, z->y, z->s_p, z->s_m, w.f, w.h, mu, &phi, &theta);
  const double theta_max = 1e4 * fmax(1.0, theta);
  const double theta_min = 1e-4 * fmax(1.0, theta);
  double dw_last = 0.0;
  int status = 10, it;
  double tau = fmax(TAU_MIN, 1.0 - mu);

  for (it = 0; it <= o->max_iter; ++it) {
    if (!isfinite(w.f) || !all_finite(w.h, m) || !all_finite(w.grad, n)) { status = 13; break; }
    /* A-2: overall convergence, eq. (infiniteOCP-outerTol) */
    double E0, E0u, Emu;
    opt_error(&w, z, 0.0, &E0, &E0u);
    info->E0_scaled = E0; info->E0_unscaled = E0u;
    if (E0 <= o->tol) { status = 0; break; }
    if (it == o->max_iter) { status = 10; break; }
    /* A-3: barrier subproblem convergence, eq. (infiniteOCP-innerTol) */
    opt_error(&w, z, mu, &Emu, NULL);
    while (Emu <= KAPPA_EPS * mu && mu > mu_min) {
      mu = fmax(mu_min, fmin(KAPPA_MU * mu, pow(mu, THETA_MU)));
      tau = fmax(TAU_MIN, 1.0 - mu);
      nf = 0;
      opt_error(&w, z, mu, &Emu, NULL);
    }
    merit_of(&w, z->y, z->s_p, z->s_m, w.f, w.h, mu, &phi, &theta);
    /* A-4: Newton direction with inertia correction (Algorithm 2, l. 6-14) */
    double dw = 0.0;
    if (factor_with_correction(&w, z, &dw_last, &dw, &info->inertia_retries)) { status = 12; break; }
    if (hy) info->cg_iters += direction_hy(&w, z, mu, &d);
    else direction(&w, z, mu, &d);
    /* fraction to the boundary */
    double ap = 1.0, ad = 1.0;
    for (int i = 0; i < n; ++i) {
      if (isfinite(w.yL[i]) && d.y[i] < 0.0) ap = fmin(ap, -tau * (z->y[i] - w.yL[i]) / d.y[i]);
      if (isfinite(w.yU[i]) && d.y[i] > 0.0) ap = fmin(ap, tau * (w.yU[i] - z->y[i]) / d.y[i]);
    }
    if (!hy) {
      ap = frac_to_boundary(z->s_p, d.s_p, tau, m, ap);
      ap = frac_to_boundary(z->s_m, d.s_m, tau, m, ap);
    }
    ad = frac_to_boundary(z->zL, d.zL, tau, n, ad);
    ad = frac_to_boundary(z->zU, d.zU, tau, n, ad);
    if (!hy) {
      ad = frac_to_boundary(z->b_p, d.b_p, tau, m, ad);
      ad = frac_to_boundary(z->b_m, d.b_m, tau, m, ad);
    }
    /* directional derivative of the barrier objective */
    double gphi = 0.0;
    for (int i = 0; i < n; ++i) {
      double g = w.grad[i];
      if (isfinite(w.yL[i])) g -= mu / (z->y[i] - w.yL[i]);
      if (isfinite(w.yU[i])) g += mu / (w.yU[i] - z->y[i]);
      gphi += g * d.y[i];
    }
    for (int r = 0; r < m && !hy; ++r) gphi -= mu * (d.s_p[r] / z->s_p[r] + d.s_m[r] / z->s_m[r]);
    /* A-5: backtracking filter line search (eq. infiniteOCP-lineSearch) */
    double amin;
    if (gphi < 0.0) {
      amin = fmin(GAMMA_THETA, GAMMA_PHI * theta / (-gphi));
      if (theta <= theta_min) amin = fmin(amin, DELTA_SW * pow(theta, S_THETA) / pow(-gphi, S_PHI));
      amin *= GAMMA_ALPHA;
    } else amin = GAMMA_ALPHA * GAMMA_THETA;
    double alpha = ap, ft = 0.0, phit = 0.0, thetat = 0.0;
    int accepted = 0, augment = 0, trials = 0;
    while (alpha >= amin) {
      ++trials;
      for (int i = 0; i < n; ++i) zt.y[i] = z->y[i] + alpha * d.y[i];
      for (int r = 0; r < m && !hy; ++r) { zt.s_p[r] = z->s_p[r] + alpha * d.s_p[r]; zt.s_m[r] = z->s_m[r] + alpha * d.s_m[r]; }
      or_eval(p, zt.y, &ft, NULL, ht, NULL, NULL, NULL);
      merit_of(&w, zt.y, zt.s_p, zt.s_m, ft, ht, mu, &phit, &thetat);
      int ok = isfinite(phit) && isfinite(thetat) && thetat <= theta_max;
      for (int q = 0; ok && q < nf; ++q) if (thetat >= filt_th[q] && phit >= filt_ph[q]) ok = 0;
      if (ok) {
        const int sw = gphi < 0.0 && alpha * pow(-gphi, S_PHI) > DELTA_SW * pow(theta, S_THETA);
        if (theta <= theta_min && sw) {
          if (phit <= phi + ETA_PHI * alpha * gphi) { accepted = 1; augment = 0; }
        } else if (thetat <= (1.0 - GAMMA_THETA) * theta || phit <= phi - GAMMA_PHI * theta) {
          accepted = 1; augment = 1;
        }
      }
      if (accepted) break;
      alpha *= 0.5;
    }
    info->ls_trials += trials;
    if (trace && it < trace_cap) {
      double* t = trace + 8 * it;
      t[0] = mu; t[1] = accepted ? alpha : 0.0; t[2] = ad; t[3] = dw; t[4] = theta; t[5] = phi; t[6] = Emu; t[7] = trials;
    }
    if (!accepted) { status = 11; break; }
    if (augment && nf < fcap) { filt_th[nf] = (1.0 - GAMMA_THETA) * theta; filt_ph[nf] = phi - GAMMA_PHI * theta; ++nf; }
    /* A-6: accept the trial point */
    for (int i = 0; i < n; ++i) {
      z->y[i] = zt.y[i];
      z->zL[i] += ad * d.zL[i];
      z->zU[i] += ad * d.zU[i];
    }
    for (int r = 0; r < m; ++r) {
      z->w_p[r] += alpha * d.w_p[r]; /* omega+, or lambda in the HyKKT form: the primal step */
      if (hy) continue;
      z->s_p[r] = zt.s_p[r]; z->s_m[r] = zt.s_m[r];
      z->w_m[r] += alpha * d.w_m[r];
      z->b_p[r] += ad * d.b_p[r]; z->b_m[r] += ad * d.b_m[r];
    }
    /* safeguard of the bound multipliers (W&B eq. (16)) */
    for (int i = 0; i < n; ++i) {
      if (isfinite(w.yL[i])) { double g = z->y[i] - w.yL[i]; z->zL[i] = fmax(fmin(z->zL[i], KAPPA_SIGMA * mu / g), mu / (KAPPA_SIGMA * g)); }
      if (isfinite(w.yU[i])) { double g = w.yU[i] - z->y[i]; z->zU[i] = fmax(fmin(z->zU[i], KAPPA_SIGMA * mu / g), mu / (KAPPA_SIGMA * g)); }
    }
    for (int r = 0; r < m && !hy; ++r) {
      z->b_p[r] = fmax(fmin(z->b_p[r], KAPPA_SIGMA * mu / z->s_p[r]), mu / (KAPPA_SIGMA * z->s_p[r]));
      z->b_m[r] = fmax(fmin(z->b_m[r], KAPPA_SIGMA * mu / z->s_m[r]), mu / (KAPPA_SIGMA * z->s_m[r]));
    }
    eval_all(&w, z->y);
  }
  info->status = status;
  info->iters = it;
  info->mu_final = mu;
  info->objective = w.f;
  info->delta_w_last = dw_last;
  free(dbuf); free(ht); free(filt_th); free(filt_ph);
  work_free(&w);
  return status;
}

void or_kkt_error(const or_problem* p, const or_options* o, const or_state* z, double mu,
                  double* E_scaled, double* E_unscaled) {
  work w;
  work_init(&w, p, o);
  eval_all(&w, z->y);
  opt_error(&w, z, mu, E_scaled, E_unscaled);
  work_free(&w);
}

int or_newton_step(const or_problem* p, const or_options* o, const or_state* z, double mu,
                   double delta_w, or_state* d) {
  work w;
  work_init(&w, p, o);
  eval_all(&w, z->y);
  assemble(&w, z, delta_w);
  int rc = kfactor(&w, 0.0);
  if (rc == 0 && o->kkt == 1) direction_hy(&w, z, mu, d);
  else if (rc == 0) direction(&w, z, mu, d);
  work_free(&w);
  return rc;
}
