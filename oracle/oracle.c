/*
 * Serial FP64 CPU oracle of the edge-based finite-volume loops.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path calls this file:
 * only the tests, the smoke check and the benchmark's CPU baseline load it.
 * It shares no code with the CUDA kernels (no headers, helpers or tables).
 *
 * Plain definitions, one edge after another, in the order the method
 * states them.  The paper (Sec. 2 and Sec. 3.1, Fig. "OP2loop") defines the
 * loop structure: a loop over the edge set that reads node data through the
 * edge->node map and increments both end nodes (OP_INC).  It does not print
 * the numerics, so the formulas below are the textbook ones chosen for the
 * edge-based solver (Sec. 2: Hydra marches with a 5-step Runge-Kutta
 * scheme):
 *
 *   Euler flux     f(q).n = (rho un, rho u un + p n, (rho E + p) un, c un)
 *   Rusanov        F = (f(qL).n + f(qR).n)/2 - s (qR - qL)/2,
 *                  s = max(|uL.n| + aL|n|, |uR.n| + aR|n|), a = sqrt(g p/rho)
 *   Green-Gauss    Graw_i += (q_i+q_j)/2 (x) n_e,  Graw_j -= same;  G = Graw/V
 *   van Albada     phi(a,b) = (a(b^2+eps) + b(a^2+eps)) / (a^2+b^2+2 eps)
 *   reconstruction qL = q_i + phi(G_i.dx, q_j-q_i)/2,
 *                  qR = q_j - phi(G_j.dx, q_j-q_i)/2
 *   residual       R_i += F_e, R_j -= F_e    (F is the flux out of i)
 *   time step      Lambda_i = sum_e s_e(q_i, q_j), dt_i = CFL V_i / Lambda_i
 *   RK stage       q = q0 - alpha_k (dt_i / V_i) R(q_prev),
 *                  alpha = (1/4, 1/6, 3/8, 1/2, 1) (Jameson's 5 stages)
 *
 * Layout (the oracle's own, node-major): q[i*6+k], G[i*18+k*3+d],
 * n[e*3+d], dx[e*3+d], edge[e*2+0] = i, edge[e*2+1] = j.
 *
 * Parity pins (tests/test_oracle_*.py): closed forms on the 8-node cube,
 * linear exactness of the gradient and the reconstruction on the lattice,
 * flux consistency and antisymmetry, global conservation, freestream,
 * finite differences and the dot-product test for the two sweeps.
 * The choices of wave-speed estimate, limiter and RK coefficients are not
 * fixed by the paper: against the paper they are parity unpinned, and are
 * pinned only by those self-consistency properties.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define NV 6   /* conserved variables per node */
#define NG 18  /* gradient values per node: 6 variables x 3 directions */

/* ---------------------------------------------------------------- pieces */

/* pressure of a conserved state */
static double pressure(const double q[NV], double gamma) {
  double rho = q[0];
  double ke = 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / rho;
  return (gamma - 1.0) * (q[4] - ke);
}

/* physical flux through the face with normal n */
void ora_euler_flux(const double q[NV], const double n[3], double gamma,
                    double f[NV]) {
  double rho = q[0];
  double un = (q[1] * n[0] + q[2] * n[1] + q[3] * n[2]) / rho;
  double p = pressure(q, gamma);
  f[0] = q[0] * un;
  f[1] = q[1] * un + p * n[0];
  f[2] = q[2] * un + p * n[1];
  f[3] = q[3] * un + p * n[2];
  f[4] = (q[4] + p) * un;
  f[5] = q[5] * un;
}

/* largest wave speed |u.n| + a|n| of one state */
double ora_wave_speed(const double q[NV], const double n[3], double gamma) {
  double rho = q[0];
  double un = (q[1] * n[0] + q[2] * n[1] + q[3] * n[2]) / rho;
  double p = pressure(q, gamma);
  double a = sqrt(gamma * p / rho);
  double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  return fabs(un) + a * nn;
}

/* Rusanov (local Lax-Friedrichs) flux; ties of the two wave speeds pick L */
void ora_rusanov(const double qL[NV], const double qR[NV], const double n[3],
                 double gamma, double F[NV]) {
  double fL[NV], fR[NV];
  ora_euler_flux(qL, n, gamma, fL);
  ora_euler_flux(qR, n, gamma, fR);
  double sL = ora_wave_speed(qL, n, gamma);
  double sR = ora_wave_speed(qR, n, gamma);
  double s = (sL >= sR) ? sL : sR;
  for (int k = 0; k < NV; k++)
    F[k] = 0.5 * (fL[k] + fR[k]) - 0.5 * s * (qR[k] - qL[k]);
}

double ora_van_albada(double a, double b, double eps) {
  return (a * (b * b + eps) + b * (a * a + eps)) / (a * a + b * b + 2.0 * eps);
}

/* limited linear reconstruction of the two face states of edge (i, j) */
void ora_reconstruct(const double qi[NV], const double qj[NV],
                     const double Gi[NG], const double Gj[NG],
                     const double dx[3], double eps, double qL[NV],
                     double qR[NV]) {
  for (int k = 0; k < NV; k++) {
    double b = qj[k] - qi[k];
    double ai = Gi[k * 3 + 0] * dx[0] + Gi[k * 3 + 1] * dx[1] + Gi[k * 3 + 2] * dx[2];
    double aj = Gj[k * 3 + 0] * dx[0] + Gj[k * 3 + 1] * dx[1] + Gj[k * 3 + 2] * dx[2];
    qL[k] = qi[k] + 0.5 * ora_van_albada(ai, b, eps);
    qR[k] = qj[k] - 0.5 * ora_van_albada(aj, b, eps);
  }
}

/* ------------------------------------------------------------- the loops */

/* first-order residual: R = sum over edges of +-F(q_i, q_j, n_e).
 * Rabs (nullable) receives sum_e |F_e,k| per node (the scale of R). */
void ora_flux1(int64_t N, int64_t E, const int32_t* edge, const double* q,
               const double* n, double gamma, double* R, double* Rabs) {
  memset(R, 0, sizeof(double) * NV * N);
  if (Rabs) memset(Rabs, 0, sizeof(double) * NV * N);
  for (int64_t e = 0; e < E; e++) {
    int64_t i = edge[2 * e], j = edge[2 * e + 1];
    double F[NV];
    ora_rusanov(q + NV * i, q + NV * j, n + 3 * e, gamma, F);
    for (int k = 0; k < NV; k++) {
      R[NV * i + k] += F[k];
      R[NV * j + k] -= F[k];
      if (Rabs) {
        Rabs[NV * i + k] += fabs(F[k]);
        Rabs[NV * j + k] += fabs(F[k]);
      }
    }
  }
}

/* Green-Gauss edge loop, unscaled: Graw.  Gabs (nullable) gets the sum of
 * the absolute values of the contributions. */
void ora_green_gauss(int64_t N, int64_t E, const int32_t* edge,
                     const double* q, const double* n, double* Graw,
                     double* Gabs) {
  memset(Graw, 0, sizeof(double) * NG * N);
  if (Gabs) memset(Gabs, 0, sizeof(double) * NG * N);
  for (int64_t e = 0; e < E; e++) {
    int64_t i = edge[2 * e], j = edge[2 * e + 1];
    for (int k = 0; k < NV; k++) {
      double qf = 0.5 * (q[NV * i + k] + q[NV * j + k]);
      for (int d = 0; d < 3; d++) {
        double c = qf * n[3 * e + d];
        Graw[NG * i + 3 * k + d] += c;
        Graw[NG * j + 3 * k + d] -= c;
        if (Gabs) {
          Gabs[NG * i + 3 * k + d] += fabs(c);
          Gabs[NG * j + 3 * k + d] += fabs(c);
        }
      }
    }
  }
}

/* direct node loop: G = Graw / V */
void ora_grad_scale(int64_t N, const double* Graw, const double* V, double* G) {
  for (int64_t i = 0; i < N; i++)
    for (int c = 0; c < NG; c++) G[NG * i + c] = Graw[NG * i + c] / V[i];
}

/* second-order residual from given q and G */
void ora_flux2(int64_t N, int64_t E, const int32_t* edge, const double* q,
               const double* G, const double* n, const double* dx,
               double gamma, double eps, double* R, double* Rabs) {
  memset(R, 0, sizeof(double) * NV * N);
  if (Rabs) memset(Rabs, 0, sizeof(double) * NV * N);
  for (int64_t e = 0; e < E; e++) {
    int64_t i = edge[2 * e], j = edge[2 * e + 1];
    double qL[NV], qR[NV], F[NV];
    ora_reconstruct(q + NV * i, q + NV * j, G + NG * i, G + NG * j, dx + 3 * e,
                    eps, qL, qR);
    ora_rusanov(qL, qR, n + 3 * e, gamma, F);
    for (int k = 0; k < NV; k++) {
      R[NV * i + k] += F[k];
      R[NV * j + k] -= F[k];
      if (Rabs) {
        Rabs[NV * i + k] += fabs(F[k]);
        Rabs[NV * j + k] += fabs(F[k]);
      }
    }
  }
}

/* full residual R(q, n): order 1 = flux1; order 2 = GG, scale, flux2.
 * G (nullable) receives the scaled gradient (N x 18). */
void ora_residual(int order, int64_t N, int64_t E, const int32_t* edge,
                  const double* q, const double* n, const double* dx,
                  const double* V, double gamma, double eps, double* G_work,
                  double* R, double* Rabs) {
  if (order == 1) {
    ora_flux1(N, E, edge, q, n, gamma, R, Rabs);
    return;
  }
  ora_green_gauss(N, E, edge, q, n, G_work, 0);
  ora_grad_scale(N, G_work, V, G_work);
  ora_flux2(N, E, edge, q, G_work, n, dx, gamma, eps, R, Rabs);
}

/* setup edge loop: Lambda_i = sum over incident edges of s_e(q_i, q_j) */
void ora_spectral_radius(int64_t N, int64_t E, const int32_t* edge,
                         const double* q, const double* n, double gamma,
                         double* Lam) {
  memset(Lam, 0, sizeof(double) * N);
  for (int64_t e = 0; e < E; e++) {
    int64_t i = edge[2 * e], j = edge[2 * e + 1];
    double sL = ora_wave_speed(q + NV * i, n + 3 * e, gamma);
    double sR = ora_wave_speed(q + NV * j, n + 3 * e, gamma);
    double s = (sL >= sR) ? sL : sR;
    Lam[i] += s;
    Lam[j] += s;
  }
}

/* local time step dt_i = CFL V_i / Lambda_i */
void ora_time_step(int64_t N, const double* V, const double* Lam, double cfl,
                   double* dt) {
  for (int64_t i = 0; i < N; i++) dt[i] = cfl * V[i] / Lam[i];
}

/* RK stage node update q = q0 - alpha (dt/V) R */
void ora_rk_update(int64_t N, const double* q0, const double* R,
                   const double* V, const double* dt, double alpha,
                   double* q) {
  for (int64_t i = 0; i < N; i++)
    for (int k = 0; k < NV; k++)
      q[NV * i + k] = q0[NV * i + k] - alpha * (dt[i] / V[i]) * R[NV * i + k];
}

/* ------------------------------------------------- block-Jacobi blocks
 * Hydra's Runge-Kutta march is block-Jacobi preconditioned (Sec. 2) and its
 * per-node blocks are inverted in a direct loop (`invjacs`, Table
 * "loopperfmpi").  The paper prints neither the block nor the scheme; the
 * reading taken here:
 *   M_i = sum over the edges e of node i of
 *           ( A(q_i, n_e) + s_e I) / 2   when i is the first end,
 *           (-A(q_i, n_e) + s_e I) / 2   when i is the second end,
 * the diagonal block of the Jacobian of the first-order Rusanov residual
 * with the wave speed s_e (of the states q_i, q_j) held fixed, where
 * A(q, n) = d(f(q).n)/dq is the Euler flux Jacobian;  P_i = M_i^{-1};
 * preconditioned stage  q = q0 - alpha sigma P_i R_i. */

/* A[r*6+c] = d (f(q).n)_r / d q_c, f as in ora_euler_flux (textbook
 * Jacobian of the conservative Euler flux with a passive scalar) */
void ora_flux_jacobian(const double q[NV], const double n[3], double gamma,
                       double A[NV * NV]) {
  double rho = q[0];
  double u[3] = {q[1] / rho, q[2] / rho, q[3] / rho};
  double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  double k = 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  double g1 = gamma - 1.0;
  double p = pressure(q, gamma);
  double H = (q[4] + p) / rho;
  double c = q[5] / rho;
  memset(A, 0, sizeof(double) * NV * NV);
  /* mass flux m.n */
  for (int b = 0; b < 3; b++) A[0 * NV + 1 + b] = n[b];
  /* momentum m_a un + p n_a */
  for (int a = 0; a < 3; a++) {
    A[(1 + a) * NV + 0] = -u[a] * un + g1 * k * n[a];
    for (int b = 0; b < 3; b++)
      A[(1 + a) * NV + 1 + b] = (a == b ? un : 0.0) + u[a] * n[b] - g1 * n[a] * u[b];
    A[(1 + a) * NV + 4] = g1 * n[a];
  }
  /* energy (E + p) un */
  A[4 * NV + 0] = un * (g1 * k - H);
  for (int b = 0; b < 3; b++) A[4 * NV + 1 + b] = H * n[b] - g1 * un * u[b];
  A[4 * NV + 4] = gamma * un;
  /* passive scalar c un */
  A[5 * NV + 0] = -c * un;
  for (int b = 0; b < 3; b++) A[5 * NV + 1 + b] = c * n[b];
  A[5 * NV + 5] = un;
}

/* M (N x 36, node-major, row-major blocks) */
void ora_jacobi_blocks(int64_t N, int64_t E, const int32_t* edge,
                       const double* q, const double* n, double gamma,
                       double* M) {
  memset(M, 0, sizeof(double) * NV * NV * N);
  for (int64_t e = 0; e < E; e++) {
    int64_t i = edge[2 * e], j = edge[2 * e + 1];
    double sL = ora_wave_speed(q + NV * i, n + 3 * e, gamma);
    double sR = ora_wave_speed(q + NV * j, n + 3 * e, gamma);
    double s = (sL >= sR) ? sL : sR;
    double Ai[NV * NV], Aj[NV * NV];
    ora_flux_jacobian(q + NV * i, n + 3 * e, gamma, Ai);
    ora_flux_jacobian(q + NV * j, n + 3 * e, gamma, Aj);
    for (int r = 0; r < NV * NV; r++) {
      M[NV * NV * i + r] += 0.5 * Ai[r];
      M[NV * NV * j + r] -= 0.5 * Aj[r];
    }
    for (int r = 0; r < NV; r++) {
      M[NV * NV * i + r * NV + r] += 0.5 * s;
      M[NV * NV * j + r * NV + r] += 0.5 * s;
    }
  }
}

/* P_i = M_i^{-1} by Gauss-Jordan elimination on [M_i | I] with partial
 * pivoting (the largest |pivot| in the column, the first on ties).
 * Returns the number of blocks with a zero pivot (their P is not finite). */
int64_t ora_block_invert(int64_t N, const double* M, double* P) {
  int64_t singular = 0;
  for (int64_t i = 0; i < N; i++) {
    double a[NV][2 * NV];
    for (int r = 0; r < NV; r++)
      for (int c = 0; c < NV; c++) {
        a[r][c] = M[NV * NV * i + r * NV + c];
        a[r][NV + c] = (r == c) ? 1.0 : 0.0;
      }
    int bad = 0;
    for (int k = 0; k < NV; k++) {
      int piv = k;
      for (int r = k + 1; r < NV; r++)
        if (fabs(a[r][k]) > fabs(a[piv][k])) piv = r;
      if (piv != k)
        for (int c = 0; c < 2 * NV; c++) {
          double t = a[k][c];
          a[k][c] = a[piv][c];
          a[piv][c] = t;
        }
      if (a[k][k] == 0.0) bad = 1;
      double inv = 1.0 / a[k][k];
      for (int c = 0; c < 2 * NV; c++) a[k][c] *= inv;
      for (int r = 0; r < NV; r++) {
        if (r == k) continue;
        double f = a[r][k];
        for (int c = 0; c < 2 * NV; c++) a[r][c] -= f * a[k][c];
      }
    }
    singular += bad;
    for (int r = 0; r < NV; r++)
      for (int c = 0; c < NV; c++) P[NV * NV * i + r * NV + c] = a[r][NV + c];
  }
  return singular;
}

/* preconditioned stage: q = q0 - alpha sigma P R, per node */
void ora_precond_update(int64_t N, const double* q0, const double* R,
                        const double* P, double alpha_sigma, double* q) {
  for (int64_t i = 0; i < N; i++)
    for (int r = 0; r < NV; r++) {
      double s = 0.0;
      for (int c = 0; c < NV; c++) s += P[NV * NV * i + r * NV + c] * R[NV * i + c];
      q[NV * i + r] = q0[NV * i + r] - alpha_sigma * s;
    }
}

/* ---------------------------------------------------------- viscous flux
 * Edge-based Navier-Stokes viscous flux (Hydra's `vfluxedge` analogue; the
 * paper names the loop, Table "loopperfmpi", but not its formula):
 *  - primitive gradients at each end from the conserved gradients G:
 *      grad u_d = (grad m_d - u_d grad rho) / rho,
 *      grad p = (gamma-1)(grad E - u . grad m + |u|^2/2 grad rho),
 *      grad T = (grad p - T grad rho) / rho   with T = p / rho,
 *      grad c = G[5] (the conserved passive scalar);
 *  - face gradient: the average of the two ends, corrected along the edge
 *      g_f = g_avg + ((phi_j - phi_i) - g_avg . dx) dx / |dx|^2,
 *    so that g_f . dx equals the jump exactly;
 *  - face velocity u_f = (u_i + u_j) / 2;
 *  - stress tau = mu (grad u + grad u^T - 2/3 div u I) (Stokes' hypothesis),
 *    heat flux coefficient kappa = mu gamma / ((gamma-1) Pr);
 *  - Fv = (0, tau n, (tau u_f) . n + kappa grad T . n, D grad c . n).
 * The residual receives -Fv at i and +Fv at j (diffusion is the negative of
 * an outgoing flux). */
static void prim_grad(const double q[NV], const double G[NG], double gamma,
                      double gu[3][3], double gT[3], double gc[3], double* T,
                      double u[3]) {
  double rho = q[0];
  for (int a = 0; a < 3; a++) u[a] = q[1 + a] / rho;
  double p = pressure(q, gamma);
  *T = p / rho;
  for (int d = 0; d < 3; d++) {
    double grho = G[d];
    for (int a = 0; a < 3; a++) gu[a][d] = (G[3 * (1 + a) + d] - u[a] * grho) / rho;
    double udm = u[0] * G[3 + d] + u[1] * G[6 + d] + u[2] * G[9 + d];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double gp = (gamma - 1.0) * (G[12 + d] - udm + 0.5 * uu * grho);
    gT[d] = (gp - (*T) * grho) / rho;
    gc[d] = G[15 + d];
  }
}

static void face_gradient(const double gi[3], const double gj[3], double jump,
                          const double dx[3], double gf[3]) {
  double dd = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
  double ga[3], gdx = 0.0;
  for (int d = 0; d < 3; d++) {
    ga[d] = 0.5 * (gi[d] + gj[d]);
    gdx += ga[d] * dx[d];
  }
  for (int d = 0; d < 3; d++) gf[d] = ga[d] + (jump - gdx) * dx[d] / dd;
}

void ora_viscous_flux(const double qi[NV], const double qj[NV],
                      const double Gi[NG], const double Gj[NG],
                      const double n[3], const double dx[3], double gamma,
                      double mu, double prandtl, double diff, double Fv[NV]) {
  double gui[3][3], guj[3][3], gTi[3], gTj[3], gci[3], gcj[3], Ti, Tj, ui[3], uj[3];
  prim_grad(qi, Gi, gamma, gui, gTi, gci, &Ti, ui);
  prim_grad(qj, Gj, gamma, guj, gTj, gcj, &Tj, uj);
  double gu[3][3], gT[3], gc[3], uf[3];
  for (int a = 0; a < 3; a++) {
    face_gradient(gui[a], guj[a], uj[a] - ui[a], dx, gu[a]);
    uf[a] = 0.5 * (ui[a] + uj[a]);
  }
  face_gradient(gTi, gTj, Tj - Ti, dx, gT);
  face_gradient(gci, gcj, qj[5] - qi[5], dx, gc);
  double div = gu[0][0] + gu[1][1] + gu[2][2];
  double tau[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++)
      tau[a][b] = mu * (gu[a][b] + gu[b][a] - (a == b ? 2.0 / 3.0 * div : 0.0));
  double kappa = mu * gamma / ((gamma - 1.0) * prandtl);
  Fv[0] = 0.0;
  Fv[4] = 0.0;
  for (int a = 0; a < 3; a++) {
    double tn = tau[a][0] * n[0] + tau[a][1] * n[1] + tau[a][2] * n[2];
    Fv[1 + a] = tn;
    Fv[4] += tn * uf[a];
  }
  Fv[4] += kappa * (gT[0] * n[0] + gT[1] * n[1] + gT[2] * n[2]);
  Fv[5] = diff * (gc[0] * n[0] + gc[1] * n[1] + gc[2] * n[2]);
}

/* viscous edge loop: R_i -= Fv, R_j += Fv (R zeroed first); Rabs gets the
 * sum of |Fv| per node */
void ora_viscous(int64_t N, int64_t E, const int32_t* edge, const double* q,
                 const double* G, const double* n, const double* dx,
                 double gamma, double mu, double prandtl, double diff,
                 double* R, double* Rabs) {
  memset(R, 0, sizeof(double) * NV * N);
  if (Rabs) memset(Rabs, 0, sizeof(double) * NV * N);
  for (int64_t e = 0; e < E; e++) {
    int64_t i = edge[2 * e], j = edge[2 * e + 1];
    double F[NV];
    ora_viscous_flux(q + NV * i, q + NV * j, G + NG * i, G + NG * j, n + 3 * e,
                     dx + 3 * e, gamma, mu, prandtl, diff, F);
    for (int k = 0; k < NV; k++) {
      R[NV * i + k] -= F[k];
      R[NV * j + k] += F[k];
      if (Rabs) {
        Rabs[NV * i + k] += fabs(F[k]);
        Rabs[NV * j + k] += fabs(F[k]);
      }
    }
  }
}

/* Global reductions over the rows of an (n x dim) node-major array, per
 * component: op 0 sum, 1 Euclidean norm sqrt(sum x^2), 2 max |x|, 3 min x
 * (the residual norms and the global time step of an explicit solver). */
void ora_reduce(int64_t n, int dim, const double* x, int op, double* out) {
  for (int k = 0; k < dim; k++) {
    double acc = (op == 3) ? INFINITY : 0.0;
    for (int64_t i = 0; i < n; i++) {
      double v = x[(int64_t)dim * i + k];
      if (op == 0) acc += v;
      else if (op == 1) acc += v * v;
      else if (op == 2) acc = fabs(v) > acc ? fabs(v) : acc;
      else acc = v < acc ? v : acc;
    }
    out[k] = (op == 1) ? sqrt(acc) : acc;
  }
}

/* 0 if every node has rho > 0 and p > 0, else 1 + the first bad node */
int64_t ora_check_state(int64_t N, const double* q, double gamma) {
  for (int64_t i = 0; i < N; i++)
    if (!(q[NV * i] > 0.0) || !(pressure(q + NV * i, gamma) > 0.0)) return 1 + i;
  return 0;
}

static const double RK_ALPHA[5] = {0.25, 1.0 / 6.0, 0.375, 0.5, 1.0};

/* explicit march: `steps` RK steps of `stages` stages (<= 5, Jameson's
 * coefficients taken from the last `stages`), dt frozen from the initial
 * state.  Work arrays: q0 (N*6), R (N*6), G (N*18), Lam (N), dt (N).
 * Returns 0, or -(1 + stage index) at the first positivity failure. */
int64_t ora_march(int order, int steps, int stages, int64_t N, int64_t E,
                  const int32_t* edge, double* q, const double* n,
                  const double* dx, const double* V, double gamma, double eps,
                  double cfl, double* q0, double* R, double* G, double* Lam,
                  double* dt) {
  ora_spectral_radius(N, E, edge, q, n, gamma, Lam);
  ora_time_step(N, V, Lam, cfl, dt);
  int64_t count = 0;
  for (int st = 0; st < steps; st++) {
    memcpy(q0, q, sizeof(double) * NV * N);
    for (int k = 0; k < stages; k++) {
      ora_residual(order, N, E, edge, q, n, dx, V, gamma, eps, G, R, 0);
      ora_rk_update(N, q0, R, V, dt, RK_ALPHA[5 - stages + k], q);
      if (ora_check_state(N, q, gamma)) return -(1 + count);
      count++;
    }
  }
  return 0;
}

/* --------------------------------------------- tangent (forward) sweep
 * Linearisation of R(q, n) in the direction (qd, nd); dx and V fixed.
 * d|x|/dx = sign(x) with sign(0) = 0; the max picks L on ties. */

static double sgn(double x) { return (x > 0.0) - (x < 0.0); }

/* one side of the Rusanov flux: f(q).n and its wave speed, with tangents */
static void side_tangent(const double q[NV], const double qd[NV],
                         const double n[3], const double nd[3], double gamma,
                         double f[NV], double fd[NV], double* lam,
                         double* lamd) {
  double rho = q[0], rhod = qd[0];
  double mn = q[1] * n[0] + q[2] * n[1] + q[3] * n[2];
  double mnd = qd[1] * n[0] + qd[2] * n[1] + qd[3] * n[2] +
               q[1] * nd[0] + q[2] * nd[1] + q[3] * nd[2];
  double un = mn / rho;
  double und = mnd / rho - un * rhod / rho;
  double mm = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  double mmd = 2.0 * (q[1] * qd[1] + q[2] * qd[2] + q[3] * qd[3]);
  double p = (gamma - 1.0) * (q[4] - 0.5 * mm / rho);
  double pd = (gamma - 1.0) *
              (qd[4] - 0.5 * mmd / rho + 0.5 * mm * rhod / (rho * rho));
  double a = sqrt(gamma * p / rho);
  double ad = gamma * pd / (2.0 * a * rho) - a * rhod / (2.0 * rho);
  double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  double nnd = (n[0] * nd[0] + n[1] * nd[1] + n[2] * nd[2]) / nn;
  *lam = fabs(un) + a * nn;
  *lamd = sgn(un) * und + ad * nn + a * nnd;
  for (int k = 0; k < NV; k++) {
    f[k] = q[k] * un;
    fd[k] = qd[k] * un + q[k] * und;
  }
  for (int d = 0; d < 3; d++) {
    f[1 + d] += p * n[d];
    fd[1 + d] += pd * n[d] + p * nd[d];
  }
  f[4] += p * un;
  fd[4] += pd * un + p * und;
}

static void rusanov_tangent(const double qL[NV], const double qLd[NV],
                            const double qR[NV], const double qRd[NV],
                            const double n[3], const double nd[3],
                            double gamma, double F[NV], double Fd[NV]) {
  double fL[NV], fLd[NV], fR[NV], fRd[NV], lL, lLd, lR, lRd;
  side_tangent(qL, qLd, n, nd, gamma, fL, fLd, &lL, &lLd);
  side_tangent(qR, qRd, n, nd, gamma, fR, fRd, &lR, &lRd);
  double s = (lL >= lR) ? lL : lR;
  double sd = (lL >= lR) ? lLd : lRd;
  for (int k = 0; k < NV; k++) {
    F[k] = 0.5 * (fL[k] + fR[k]) - 0.5 * s * (qR[k] - qL[k]);
    Fd[k] = 0.5 * (fLd[k] + fRd[k]) - 0.5 * sd * (qR[k] - qL[k]) -
            0.5 * s * (qRd[k] - qLd[k]);
  }
}

/* partial derivatives of the van Albada function */
static void van_albada_partials(double a, double b, double eps, double* phi,
                                double* pa, double* pb) {
  double num = a * (b * b + eps) + b * (a * a + eps);
  double den = a * a + b * b + 2.0 * eps;
  *phi = num / den;
  *pa = (b * b + eps + 2.0 * a * b - 2.0 * a * (*phi)) / den;
  *pb = (a * a + eps + 2.0 * a * b - 2.0 * b * (*phi)) / den;
}

void ora_residual_tangent(int order, int64_t N, int64_t E,
                          const int32_t* edge, const double* q,
                          const double* n, const double* dx, const double* V,
                          double gamma, double eps, const double* qd,
                          const double* nd, double* G, double* Gd,
                          double* Rd) {
  memset(Rd, 0, sizeof(double) * NV * N);
  if (order == 2) {
    /* gradient and its tangent */
    memset(G, 0, sizeof(double) * NG * N);
    memset(Gd, 0, sizeof(double) * NG * N);
    for (int64_t e = 0; e < E; e++) {
      int64_t i = edge[2 * e], j = edge[2 * e + 1];
      for (int k = 0; k < NV; k++) {
        double qf = 0.5 * (q[NV * i + k] + q[NV * j + k]);
        double qfd = 0.5 * (qd[NV * i + k] + qd[NV * j + k]);
        for (int d = 0; d < 3; d++) {
          double c = qf * n[3 * e + d];
          double cd = qfd * n[3 * e + d] + qf * nd[3 * e + d];
          G[NG * i + 3 * k + d] += c;
          G[NG * j + 3 * k + d] -= c;
          Gd[NG * i + 3 * k + d] += cd;
          Gd[NG * j + 3 * k + d] -= cd;
        }
      }
    }
    for (int64_t i = 0; i < N; i++)
      for (int c = 0; c < NG; c++) {
        G[NG * i + c] /= V[i];
        Gd[NG * i + c] /= V[i];
      }
  }
  for (int64_t e = 0; e < E; e++) {
    int64_t i = edge[2 * e], j = edge[2 * e + 1];
    const double *qi = q + NV * i, *qj = q + NV * j;
    const double *qid = qd + NV * i, *qjd = qd + NV * j;
    double qL[NV], qR[NV], qLd[NV], qRd[NV], F[NV], Fd[NV];
    if (order == 1) {
      for (int k = 0; k < NV; k++) {
        qL[k] = qi[k]; qLd[k] = qid[k];
        qR[k] = qj[k]; qRd[k] = qjd[k];
      }
    } else {
      const double *Gi = G + NG * i, *Gj = G + NG * j;
      const double *Gid = Gd + NG * i, *Gjd = Gd + NG * j;
      const double* x = dx + 3 * e;
      for (int k = 0; k < NV; k++) {
        double b = qj[k] - qi[k], bd = qjd[k] - qid[k];
        double ai = Gi[3 * k] * x[0] + Gi[3 * k + 1] * x[1] + Gi[3 * k + 2] * x[2];
        double aid = Gid[3 * k] * x[0] + Gid[3 * k + 1] * x[1] + Gid[3 * k + 2] * x[2];
        double aj = Gj[3 * k] * x[0] + Gj[3 * k + 1] * x[1] + Gj[3 * k + 2] * x[2];
        double ajd = Gjd[3 * k] * x[0] + Gjd[3 * k + 1] * x[1] + Gjd[3 * k + 2] * x[2];
        double phi, pa, pb, phj, paj, pbj;
        van_albada_partials(ai, b, eps, &phi, &pa, &pb);
        van_albada_partials(aj, b, eps, &phj, &paj, &pbj);
        qL[k] = qi[k] + 0.5 * phi;
        qLd[k] = qid[k] + 0.5 * (pa * aid + pb * bd);
        qR[k] = qj[k] - 0.5 * phj;
        qRd[k] = qjd[k] - 0.5 * (paj * ajd + pbj * bd);
      }
    }
    rusanov_tangent(qL, qLd, qR, qRd, n + 3 * e, nd + 3 * e, gamma, F, Fd);
    for (int k = 0; k < NV; k++) {
      Rd[NV * i + k] += Fd[k];
      Rd[NV * j + k] -= Fd[k];
    }
  }
}

/* --------------------------------------------- reverse (adjoint) sweep
 * J = lam . R(q, n) = sum_e (lam_i - lam_j) . F_e.  Outputs qb = dJ/dq
 * (N x 6) and nb = dJ/dn (E x 3).  Work: G (N*18), Gb (N*18). */

/* reverse of one side: given fb (adjoint of f) and lamb (adjoint of the
 * wave speed), accumulate into qb (6) and nb (3) */
static void side_reverse(const double q[NV], const double n[3], double gamma,
                         const double fb[NV], double lamb, double qb[NV],
                         double nb[3]) {
  double rho = q[0];
  double mn = q[1] * n[0] + q[2] * n[1] + q[3] * n[2];
  double un = mn / rho;
  double mm = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  double p = (gamma - 1.0) * (q[4] - 0.5 * mm / rho);
  double a = sqrt(gamma * p / rho);
  double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  /* forward: lam = |un| + a nn;  f_k = q_k un (+ p n_d, + p un) */
  double unb = sgn(un) * lamb;
  double ab = lamb * nn;
  double nnb = lamb * a;
  double pb = 0.0;
  for (int k = 0; k < NV; k++) {
    qb[k] += fb[k] * un;
    unb += fb[k] * q[k];
  }
  for (int d = 0; d < 3; d++) {
    pb += fb[1 + d] * n[d];
    nb[d] += fb[1 + d] * p;
  }
  pb += fb[4] * un;
  unb += fb[4] * p;
  /* nn = |n| */
  for (int d = 0; d < 3; d++) nb[d] += nnb * n[d] / nn;
  /* a = sqrt(gamma p / rho) */
  pb += ab * gamma / (2.0 * a * rho);
  double rhob = -ab * a / (2.0 * rho);
  /* p = (gamma-1)(q4 - mm/(2 rho)) */
  qb[4] += (gamma - 1.0) * pb;
  for (int d = 0; d < 3; d++) qb[1 + d] -= (gamma - 1.0) * pb * q[1 + d] / rho;
  rhob += (gamma - 1.0) * pb * 0.5 * mm / (rho * rho);
  /* un = mn / rho */
  for (int d = 0; d < 3; d++) {
    qb[1 + d] += unb * n[d] / rho;
    nb[d] += unb * q[1 + d] / rho;
  }
  rhob -= unb * un / rho;
  qb[0] += rhob;
}

/* reverse of the Rusanov flux with adjoint weights w = dJ/dF */
static void rusanov_reverse(const double qL[NV], const double qR[NV],
                            const double n[3], double gamma,
                            const double w[NV], double qLb[NV], double qRb[NV],
                            double nb[3]) {
  double sL = ora_wave_speed(qL, n, gamma);
  double sR = ora_wave_speed(qR, n, gamma);
  double s = (sL >= sR) ? sL : sR;
  double fb[NV], sb = 0.0;
  for (int k = 0; k < NV; k++) {
    fb[k] = 0.5 * w[k];
    sb -= 0.5 * w[k] * (qR[k] - qL[k]);
    qRb[k] -= 0.5 * s * w[k];
    qLb[k] += 0.5 * s * w[k];
  }
  double lLb = (sL >= sR) ? sb : 0.0;
  double lRb = (sL >= sR) ? 0.0 : sb;
  side_reverse(qL, n, gamma, fb, lLb, qLb, nb);
  side_reverse(qR, n, gamma, fb, lRb, qRb, nb);
}

void ora_residual_reverse(int order, int64_t N, int64_t E,
                          const int32_t* edge, const double* q,
                          const double* n, const double* dx, const double* V,
                          double gamma, double eps, const double* lam,
                          double* G, double* Gb, double* qb, double* nb) {
  memset(qb, 0, sizeof(double) * NV * N);
  memset(nb, 0, sizeof(double) * 3 * E);
  if (order == 2) {
    ora_green_gauss(N, E, edge, q, n, G, 0);
    ora_grad_scale(N, G, V, G);
    memset(Gb, 0, sizeof(double) * NG * N);
  }
  /* flux edge loop, reversed */
  for (int64_t e = 0; e < E; e++) {
    int64_t i = edge[2 * e], j = edge[2 * e + 1];
    const double *qi = q + NV * i, *qj = q + NV * j;
    double w[NV];
    for (int k = 0; k < NV; k++) w[k] = lam[NV * i + k] - lam[NV * j + k];
    double qL[NV], qR[NV], qLb[NV] = {0}, qRb[NV] = {0};
    if (order == 1) {
      for (int k = 0; k < NV; k++) { qL[k] = qi[k]; qR[k] = qj[k]; }
    } else {
      ora_reconstruct(qi, qj, G + NG * i, G + NG * j, dx + 3 * e, eps, qL, qR);
    }
    rusanov_reverse(qL, qR, n + 3 * e, gamma, w, qLb, qRb, nb + 3 * e);
    if (order == 1) {
      for (int k = 0; k < NV; k++) {
        qb[NV * i + k] += qLb[k];
        qb[NV * j + k] += qRb[k];
      }
      continue;
    }
    const double *Gi = G + NG * i, *Gj = G + NG * j;
    const double* x = dx + 3 * e;
    for (int k = 0; k < NV; k++) {
      double b = qj[k] - qi[k];
      double ai = Gi[3 * k] * x[0] + Gi[3 * k + 1] * x[1] + Gi[3 * k + 2] * x[2];
      double aj = Gj[3 * k] * x[0] + Gj[3 * k + 1] * x[1] + Gj[3 * k + 2] * x[2];
      double phi, pa, pb, phj, paj, pbj;
      van_albada_partials(ai, b, eps, &phi, &pa, &pb);
      van_albada_partials(aj, b, eps, &phj, &paj, &pbj);
      /* qL = qi + phi/2 ; qR = qj - phj/2 */
      qb[NV * i + k] += qLb[k];
      qb[NV * j + k] += qRb[k];
      double phib = 0.5 * qLb[k];
      double phjb = -0.5 * qRb[k];
      double aib = phib * pa, ajb = phjb * paj;
      double bb = phib * pb + phjb * pbj;
      /* b = qj - qi */
      qb[NV * j + k] += bb;
      qb[NV * i + k] -= bb;
      /* ai = Gi[k].dx, aj = Gj[k].dx */
      for (int d = 0; d < 3; d++) {
        Gb[NG * i + 3 * k + d] += aib * x[d];
        Gb[NG * j + 3 * k + d] += ajb * x[d];
      }
    }
  }
  if (order == 1) return;
  /* scaling G = Graw / V, reversed */
  for (int64_t i = 0; i < N; i++)
    for (int c = 0; c < NG; c++) Gb[NG * i + c] /= V[i];
  /* Green-Gauss edge loop, reversed */
  for (int64_t e = 0; e < E; e++) {
    int64_t i = edge[2 * e], j = edge[2 * e + 1];
    for (int k = 0; k < NV; k++) {
      double qf = 0.5 * (q[NV * i + k] + q[NV * j + k]);
      double qfb = 0.0;
      for (int d = 0; d < 3; d++) {
        double cb = Gb[NG * i + 3 * k + d] - Gb[NG * j + 3 * k + d];
        qfb += cb * n[3 * e + d];
        nb[3 * e + d] += cb * qf;
      }
      qb[NV * i + k] += 0.5 * qfb;
      qb[NV * j + k] += 0.5 * qfb;
    }
  }
}

/* per-edge distance to the non-differentiable points: min(|uL.n|, |uR.n|,
 * |sL - sR|) of the face states (used to keep finite differences away) */
void ora_kink_margin(int order, int64_t N, int64_t E, const int32_t* edge,
                     const double* q, const double* n, const double* dx,
                     const double* V, double gamma, double eps, double* G,
                     double* margin) {
  if (order == 2) {
    ora_green_gauss(N, E, edge, q, n, G, 0);
    ora_grad_scale(N, G, V, G);
  }
  for (int64_t e = 0; e < E; e++) {
    int64_t i = edge[2 * e], j = edge[2 * e + 1];
    double qL[NV], qR[NV];
    if (order == 1) {
      for (int k = 0; k < NV; k++) { qL[k] = q[NV * i + k]; qR[k] = q[NV * j + k]; }
    } else {
      ora_reconstruct(q + NV * i, q + NV * j, G + NG * i, G + NG * j,
                      dx + 3 * e, eps, qL, qR);
    }
    const double* ne = n + 3 * e;
    double unL = (qL[1] * ne[0] + qL[2] * ne[1] + qL[3] * ne[2]) / qL[0];
    double unR = (qR[1] * ne[0] + qR[2] * ne[1] + qR[3] * ne[2]) / qR[0];
    double m = fabs(unL);
    if (fabs(unR) < m) m = fabs(unR);
    double ds = fabs(ora_wave_speed(qL, ne, gamma) - ora_wave_speed(qR, ne, gamma));
    if (ds < m) m = ds;
    margin[e] = m;
  }
}

/* ------------------------------------------------- march derivatives
 * The explicit march with a given, fixed local time step dt (Sec. 2: the
 * 5-step Runge-Kutta scheme; dt frozen, so it is an input and not
 * differentiated).  Step n, with D = diag(dt/V):
 *   s_0 = q^n,  s_k = q^n - alpha_k D R(s_{k-1})  (k = 1..stages),
 *   q^{n+1} = s_stages.
 * Tangent (directions qd of q^0 and nd of the normals):
 *   sd_0 = qd^n,  sd_k = qd^n - alpha_k D (dR/dq(s_{k-1}) sd_{k-1} + dR/dn nd).
 * Reverse, for J = g . q^N: with sb_stages = qbar^{n+1},
 *   lam_k = -alpha_k D sb_k,  sb_{k-1} = dR/dq(s_{k-1})^T lam_k,
 *   nbar += dR/dn(s_{k-1})^T lam_k,  qbar^n = sum_{k>=1} sb_k + sb_0. */
static double rk_alpha(int stages, int k) { return RK_ALPHA[5 - stages + k]; }

/* q advanced by `steps` steps in place; returns 0 or -(1 + stage) when a
 * state loses positivity.  Work: q0, R (N x 6), G (N x 18). */
int64_t ora_march_dt(int order, int steps, int stages, int64_t N, int64_t E,
                     const int32_t* edge, double* q, const double* n,
                     const double* dx, const double* V, double gamma,
                     double eps, const double* dt, double* q0, double* R,
                     double* G) {
  int64_t count = 0;
  for (int st = 0; st < steps; st++) {
    memcpy(q0, q, sizeof(double) * NV * N);
    for (int k = 0; k < stages; k++) {
      ora_residual(order, N, E, edge, q, n, dx, V, gamma, eps, G, R, 0);
      ora_rk_update(N, q0, R, V, dt, rk_alpha(stages, k), q);
      if (ora_check_state(N, q, gamma)) return -(1 + count);
      count++;
    }
  }
  return 0;
}

/* q and qd advanced together (qd in/out).  Work: q0, qd0, R, Rd (N x 6),
 * G, Gd (N x 18). */
void ora_march_tangent(int order, int steps, int stages, int64_t N, int64_t E,
                       const int32_t* edge, double* q, const double* n,
                       const double* dx, const double* V, double gamma,
                       double eps, const double* dt, double* qd,
                       const double* nd, double* q0, double* qd0, double* R,
                       double* Rd, double* G, double* Gd) {
  for (int st = 0; st < steps; st++) {
    memcpy(q0, q, sizeof(double) * NV * N);
    memcpy(qd0, qd, sizeof(double) * NV * N);
    for (int k = 0; k < stages; k++) {
      double a = rk_alpha(stages, k);
      ora_residual_tangent(order, N, E, edge, q, n, dx, V, gamma, eps, qd, nd,
                           G, Gd, Rd);
      ora_residual(order, N, E, edge, q, n, dx, V, gamma, eps, G, R, 0);
      ora_rk_update(N, qd0, Rd, V, dt, a, qd);
      ora_rk_update(N, q0, R, V, dt, a, q);
    }
  }
}

/* Reverse sweep.  q: the initial state (not modified); g: qbar at the end
 * on entry, qbar^0 on return; nbar (E x 3) receives dJ/dn.  S holds every
 * stage's input state (steps * stages * N * 6 doubles); work: q0, R, lam,
 * qb, acc (N x 6), G, Gb (N x 18), nb (E x 3). */
void ora_march_reverse(int order, int steps, int stages, int64_t N, int64_t E,
                       const int32_t* edge, const double* q, const double* n,
                       const double* dx, const double* V, double gamma,
                       double eps, const double* dt, double* g, double* nbar,
                       double* S, double* q0, double* R, double* lam,
                       double* qb, double* acc, double* G, double* Gb,
                       double* nb) {
  const int64_t sz = NV * N;
  /* forward, keeping s_{k-1} of every stage */
  double* s = S;
  memcpy(s, q, sizeof(double) * sz);
  for (int st = 0; st < steps; st++) {
    const double* qn = S + (int64_t)st * stages * sz;
    for (int k = 0; k < stages; k++) {
      const double* sk = S + ((int64_t)st * stages + k) * sz;
      ora_residual(order, N, E, edge, sk, n, dx, V, gamma, eps, G, R, 0);
      double* next = (st == steps - 1 && k == stages - 1)
                         ? q0
                         : S + ((int64_t)st * stages + k + 1) * sz;
      ora_rk_update(N, qn, R, V, dt, rk_alpha(stages, k), next);
    }
  }
  memset(nbar, 0, sizeof(double) * 3 * E);
  /* reverse: g holds sb_stages of the current step */
  for (int st = steps - 1; st >= 0; st--) {
    memset(acc, 0, sizeof(double) * sz);
    for (int k = stages - 1; k >= 0; k--) {
      const double* sk = S + ((int64_t)st * stages + k) * sz; /* s_{k}, input of stage k+1 */
      double a = rk_alpha(stages, k);
      for (int64_t i = 0; i < N; i++)
        for (int c = 0; c < NV; c++) {
          acc[NV * i + c] += g[NV * i + c];
          lam[NV * i + c] = -a * (dt[i] / V[i]) * g[NV * i + c];
        }
      ora_residual_reverse(order, N, E, edge, sk, n, dx, V, gamma, eps, lam, G,
                           Gb, qb, nb);
      for (int64_t e = 0; e < 3 * E; e++) nbar[e] += nb[e];
      memcpy(g, qb, sizeof(double) * sz);
    }
    for (int64_t i = 0; i < sz; i++) g[i] += acc[i];
  }
}

/* ------------------------------------------------ node-limited scheme
 * The alternative to the van Albada edge limiter: limiters of the
 * Barth-Jespersen (1989) and Venkatakrishnan (1995) type, which limit each
 * node's gradient once for all its edges.  The paper does not say which
 * limiter Hydra uses; these are the two textbook node limiters.
 *
 *   qmin_i, qmax_i   min / max of q over node i and its edge neighbours
 *   per edge end (node i of edge e, d = dx at the first end, -dx at the
 *   second):  D2 = (G_i . d) / 2   (unlimited extrapolation to the edge
 *   midpoint),  D1 = qmax_i - q_i if D2 > 0, qmin_i - q_i if D2 < 0;
 *   Barth-Jespersen  phi_e = min(1, D1 / D2),
 *   Venkatakrishnan  phi_e = (D1^2 + eps2 + 2 D1 D2) / (D1^2 + 2 D2^2 + D1 D2 + eps2),
 *   and phi_e = 1 when D2 = 0;
 *   phi_i = min over the edge ends at i (1 for a node with no edges).
 *   Face states q_i + phi_i D2 at both ends, then the Rusanov flux. */
#define ORA_LIM_BJ 1
#define ORA_LIM_VENKAT 2

void ora_minmax(int64_t N, int64_t E, const int32_t* edge, const double* q,
                double* qmin, double* qmax) {
  memcpy(qmin, q, sizeof(double) * NV * N);
  memcpy(qmax, q, sizeof(double) * NV * N);
  for (int64_t e = 0; e < E; e++) {
    int64_t a = edge[2 * e], b = edge[2 * e + 1];
    for (int s = 0; s < 2; s++) {
      int64_t i = s ? b : a, j = s ? a : b;
      for (int k = 0; k < NV; k++) {
        double v = q[NV * j + k];
        if (v < qmin[NV * i + k]) qmin[NV * i + k] = v;
        if (v > qmax[NV * i + k]) qmax[NV * i + k] = v;
      }
    }
  }
}

/* half the extrapolation of variable k from node i along d */
static double half_extrap(const double* Gi, int k, const double d[3]) {
  return 0.5 * (Gi[3 * k] * d[0] + Gi[3 * k + 1] * d[1] + Gi[3 * k + 2] * d[2]);
}

double ora_limiter_edge(int kind, double d1, double d2, double eps2) {
  if (d2 == 0.0) return 1.0;
  if (kind == ORA_LIM_BJ) {
    double r = d1 / d2;
    return r < 1.0 ? r : 1.0;
  }
  return (d1 * d1 + eps2 + 2.0 * d1 * d2) / (d1 * d1 + 2.0 * d2 * d2 + d1 * d2 + eps2);
}

void ora_limiter(int kind, int64_t N, int64_t E, const int32_t* edge,
                 const double* q, const double* G, const double* dx,
                 const double* qmin, const double* qmax, double eps2,
                 double* phi) {
  for (int64_t i = 0; i < NV * N; i++) phi[i] = INFINITY;
  for (int64_t e = 0; e < E; e++) {
    for (int s = 0; s < 2; s++) {
      int64_t i = edge[2 * e + s];
      double d[3];
      for (int c = 0; c < 3; c++) d[c] = s ? -dx[3 * e + c] : dx[3 * e + c];
      for (int k = 0; k < NV; k++) {
        double d2 = half_extrap(G + NG * i, k, d);
        double d1 = d2 > 0.0 ? qmax[NV * i + k] - q[NV * i + k]
                             : qmin[NV * i + k] - q[NV * i + k];
        double f = ora_limiter_edge(kind, d1, d2, eps2);
        if (f < phi[NV * i + k]) phi[NV * i + k] = f;
      }
    }
  }
  for (int64_t i = 0; i < NV * N; i++)
    if (phi[i] == INFINITY) phi[i] = 1.0;
}

/* flux with node-limited reconstruction: R_i += F, R_j -= F */
void ora_flux2_phi(int64_t N, int64_t E, const int32_t* edge, const double* q,
                   const double* G, const double* phi, const double* n,
                   const double* dx, double gamma, double* R, double* Rabs) {
  memset(R, 0, sizeof(double) * NV * N);
  if (Rabs) memset(Rabs, 0, sizeof(double) * NV * N);
  for (int64_t e = 0; e < E; e++) {
    int64_t i = edge[2 * e], j = edge[2 * e + 1];
    const double* d = dx + 3 * e;
    double md[3] = {-d[0], -d[1], -d[2]};
    double qL[NV], qR[NV], F[NV];
    for (int k = 0; k < NV; k++) {
      qL[k] = q[NV * i + k] + phi[NV * i + k] * half_extrap(G + NG * i, k, d);
      qR[k] = q[NV * j + k] + phi[NV * j + k] * half_extrap(G + NG * j, k, md);
    }
    ora_rusanov(qL, qR, n + 3 * e, gamma, F);
    for (int k = 0; k < NV; k++) {
      R[NV * i + k] += F[k];
      R[NV * j + k] -= F[k];
      if (Rabs) {
        Rabs[NV * i + k] += fabs(F[k]);
        Rabs[NV * j + k] += fabs(F[k]);
      }
    }
  }
}

/* the whole node-limited residual: gradients, min/max, limiter, flux */
void ora_residual_limited(int kind, int64_t N, int64_t E, const int32_t* edge,
                          const double* q, const double* n, const double* dx,
                          const double* V, double gamma, double eps2, double* G,
                          double* qmin, double* qmax, double* phi, double* R,
                          double* Rabs) {
  ora_green_gauss(N, E, edge, q, n, G, 0);
  ora_grad_scale(N, G, V, G);
  ora_minmax(N, E, edge, q, qmin, qmax);
  ora_limiter(kind, N, E, edge, q, G, dx, qmin, qmax, eps2, phi);
  ora_flux2_phi(N, E, edge, q, G, phi, n, dx, gamma, R, Rabs);
}
