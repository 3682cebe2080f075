/*
 * Oracle: a plain, slow, FP64 CPU restatement of the motion-compensated
 * cone-beam backprojection of arXiv 2401.09283 and of its derivatives.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * Conventions (readings of the paper, each one listed in the design notes):
 *   - world coordinates in mm; voxel (i,j,k) sits at origin + (i,j,k)*spacing;
 *     volumes are stored [nz][ny][nx] (x fastest);
 *   - projections are stored [V][nv][nu] (u fastest); integer detector
 *     coordinates are pixel centres; samples outside the detector read 0;
 *   - projection matrices are 3x4 row-major; (u,v,w) = P * (x,y,z,1);
 *   - rigid motion (Eq. 1): T(theta) = [[R t],[0 1]] with
 *     theta = (tx,ty,tz,rx,ry,rz) in mm and rad and R = Rz(rz) Ry(ry) Rx(rx);
 *   - a view with w <= 0 at a voxel contributes nothing there.
 *
 * Everything is written as the direct loop over voxels and views that the
 * defining equation states; no blocking, fusion or reordering.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#define ORC_WEIGHT_NONE 0 /* Eq. 3 literally: sum of interpolated samples */
#define ORC_WEIGHT_FDK 1  /* c_j * (sid / w)^2 per sample                 */
#define ORC_DERIV_CENTRAL 0 /* Sec. II-B.2: central-difference gradient images */
#define ORC_DERIV_BILINEAR_EXACT 1 /* exact partials of the bilinear interpolant */

/* ---------------------------------------------------------------- 3x3 / 4x4 */

static void mat3_mul(const double A[9], const double B[9], double C[9]) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[3 * r + k] * B[3 * k + c];
      C[3 * r + c] = s;
    }
}

static void rot_x(double a, double R[9], int deriv) {
  double c = cos(a), s = sin(a);
  double M[9] = {1, 0, 0, 0, c, -s, 0, s, c};
  double D[9] = {0, 0, 0, 0, -s, -c, 0, c, -s};
  memcpy(R, deriv ? D : M, sizeof M);
}
static void rot_y(double a, double R[9], int deriv) {
  double c = cos(a), s = sin(a);
  double M[9] = {c, 0, s, 0, 1, 0, -s, 0, c};
  double D[9] = {-s, 0, c, 0, 0, 0, -c, 0, -s};
  memcpy(R, deriv ? D : M, sizeof M);
}
static void rot_z(double a, double R[9], int deriv) {
  double c = cos(a), s = sin(a);
  double M[9] = {c, -s, 0, s, c, 0, 0, 0, 1};
  double D[9] = {-s, -c, 0, c, -s, 0, 0, 0, 0};
  memcpy(R, deriv ? D : M, sizeof M);
}

/* R = Rz(rz) Ry(ry) Rx(rx); with dmask bit m set (m = 0,1,2 for x,y,z) the
 * corresponding factor is replaced by its derivative. */
static void rot_zyx(const double th[6], int dx, int dy, int dz, double R[9]) {
  double X[9], Y[9], Z[9], ZY[9];
  rot_x(th[3], X, dx);
  rot_y(th[4], Y, dy);
  rot_z(th[5], Z, dz);
  mat3_mul(Z, Y, ZY);
  mat3_mul(ZY, X, R);
}

/* Eq. 1: the 4x4 rigid transform T(theta), row-major. */
void orc_rigid(const double th[6], double T[16]) {
  double R[9];
  rot_zyx(th, 0, 0, 0, R);
  memset(T, 0, 16 * sizeof(double));
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) T[4 * r + c] = R[3 * r + c];
    T[4 * r + 3] = th[r];
  }
  T[15] = 1.0;
}

/* dT/dtheta_m for m = 0..5, written as six 4x4 row-major matrices. */
void orc_rigid_grad(const double th[6], double dT[96]) {
  memset(dT, 0, 96 * sizeof(double));
  for (int m = 0; m < 3; ++m) dT[16 * m + 4 * m + 3] = 1.0; /* translations */
  for (int m = 3; m < 6; ++m) {
    double R[9];
    rot_zyx(th, m == 3, m == 4, m == 5, R);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) dT[16 * m + 4 * r + c] = R[3 * r + c];
  }
}

/* 3x4 times 4x4. */
static void mat34_mul44(const double P[12], const double T[16], double O[12]) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += P[4 * r + k] * T[4 * k + c];
      O[4 * r + c] = s;
    }
}

/* Eq. 1 for every view: Phat_j = P_j T(theta_j).  theta may be NULL
 * (identity motion, Phat = P copied exactly). */
void orc_compose(int V, const double* P, const double* theta, double* Phat) {
  for (int j = 0; j < V; ++j) {
    if (!theta) {
      memcpy(Phat + 12 * j, P + 12 * j, 12 * sizeof(double));
      continue;
    }
    double T[16];
    orc_rigid(theta + 6 * j, T);
    mat34_mul44(P + 12 * j, T, Phat + 12 * j);
  }
}

/* ------------------------------------------------------------- sampling */

/* Detector value at integer pixel (a,b); 0 outside the detector. */
static double tap(const double* d, int nu, int nv, long a, long b) {
  if (a < 0 || b < 0 || a >= nu || b >= nv) return 0.0;
  return d[(size_t)b * nu + (size_t)a];
}

typedef struct {
  long iu, iv;    /* floor of the detector coordinate */
  double fu, fv;  /* fractional parts in [0,1) */
  int inside;     /* 0 when the coordinate is so far out that every tap is 0 */
} orc_loc;

static orc_loc locate(double ub, double vb, int nu, int nv) {
  orc_loc L;
  L.inside = (ub > -2.0 && vb > -2.0 && ub < nu + 1.0 && vb < nv + 1.0);
  if (!L.inside) {
    L.iu = L.iv = 0;
    L.fu = L.fv = 0.0;
    return L;
  }
  double fu = floor(ub), fv = floor(vb);
  L.iu = (long)fu;
  L.iv = (long)fv;
  L.fu = ub - fu;
  L.fv = vb - fv;
  return L;
}

/* Bilinear interpolation of image d at a located position (Sec. II-B.2). */
static double bilerp(const double* d, int nu, int nv, orc_loc L) {
  if (!L.inside) return 0.0;
  double d00 = tap(d, nu, nv, L.iu, L.iv), d10 = tap(d, nu, nv, L.iu + 1, L.iv);
  double d01 = tap(d, nu, nv, L.iu, L.iv + 1), d11 = tap(d, nu, nv, L.iu + 1, L.iv + 1);
  return (1 - L.fu) * (1 - L.fv) * d00 + L.fu * (1 - L.fv) * d10 + (1 - L.fu) * L.fv * d01 +
         L.fu * L.fv * d11;
}

/* ----------------------------------------------------------- forward, Eq. 3 */

typedef struct {
  int nx, ny, nz;
  double sx, sy, sz; /* spacing, mm */
  double ox, oy, oz; /* origin (centre of voxel 0,0,0), mm */
} orc_vol;

static void voxel_pos(const orc_vol* g, int i, int j, int k, double p[4]) {
  p[0] = g->ox + i * g->sx;
  p[1] = g->oy + j * g->sy;
  p[2] = g->oz + k * g->sz;
  p[3] = 1.0;
}

/* I(p) = sum_j c_j * omega_j(p) * d_j(u/w, v/w), (u,v,w) = Phat_j p~ (Eq. 3).
 * omega = 1 (NONE) or (sid/w)^2 (FDK); c_j = view_weight[j] or 1. */
void orc_bp_forward(int V, const double* Phat, const double* proj, int nu, int nv,
                    const double* view_weight, int weight_mode, double sid,
                    const orc_vol* g, double* vol) {
  const size_t img = (size_t)nu * nv;
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = 0; k < g->nz; ++k)
    for (int jy = 0; jy < g->ny; ++jy)
      for (int i = 0; i < g->nx; ++i) {
        double p[4];
        voxel_pos(g, i, jy, k, p);
        double acc = 0.0;
        for (int j = 0; j < V; ++j) {
          const double* M = Phat + 12 * j;
          double u = M[0] * p[0] + M[1] * p[1] + M[2] * p[2] + M[3];
          double v = M[4] * p[0] + M[5] * p[1] + M[6] * p[2] + M[7];
          double w = M[8] * p[0] + M[9] * p[1] + M[10] * p[2] + M[11];
          if (!(w > 0.0)) continue;
          orc_loc L = locate(u / w, v / w, nu, nv);
          double val = bilerp(proj + img * j, nu, nv, L);
          double c = view_weight ? view_weight[j] : 1.0;
          double om = (weight_mode == ORC_WEIGHT_FDK) ? (sid / w) * (sid / w) : 1.0;
          acc += c * om * val;
        }
        vol[((size_t)k * g->ny + jy) * g->nx + i] = acc;
      }
}

/* ------------------------------------------------------ VJP, Eqs. 4 and 5 */

/* Gradient images of one view along u and v: second-order central
 * differences in the interior, one-sided first differences at the two
 * edges, in units of value per pixel (Sec. II-B.2). */
void orc_gradient_images(const double* d, int nu, int nv, double* gu, double* gv) {
  for (int b = 0; b < nv; ++b)
    for (int a = 0; a < nu; ++a) {
      double x;
      if (nu < 2) x = 0.0;
      else if (a == 0) x = d[(size_t)b * nu + 1] - d[(size_t)b * nu];
      else if (a == nu - 1) x = d[(size_t)b * nu + a] - d[(size_t)b * nu + a - 1];
      else x = 0.5 * (d[(size_t)b * nu + a + 1] - d[(size_t)b * nu + a - 1]);
      gu[(size_t)b * nu + a] = x;
      double y;
      if (nv < 2) y = 0.0;
      else if (b == 0) y = d[(size_t)nu + a] - d[a];
      else if (b == nv - 1) y = d[(size_t)b * nu + a] - d[(size_t)(b - 1) * nu + a];
      else y = 0.5 * (d[(size_t)(b + 1) * nu + a] - d[(size_t)(b - 1) * nu + a]);
      gv[(size_t)b * nu + a] = y;
    }
}

/* Vector-Jacobian products of the forward above for an upstream gradient
 * dL_dvol:
 *   dL_dPhat[j] (3x4) = sum_p delta(p) * c_j * d(omega * d_j(u/w,v/w))/dPhat_j,
 * with the derivative of the interpolated sample given by Eq. 4/5 (g_u, g_v
 * per the deriv mode) and, in FDK mode, the derivative of omega = (sid/w)^2,
 * -2 omega / w, added to the third row;
 *   dL_dproj[j][b][a] = sum_p delta(p) * c_j * omega * (bilinear weight of
 * pixel (a,b) at p)   (the adjoint of Eq. 3 with respect to the data).
 * Either output may be NULL. */
void orc_bp_vjp(int V, const double* Phat, const double* proj, int nu, int nv,
                const double* view_weight, int weight_mode, int deriv_mode, double sid,
                const orc_vol* g, const double* dL_dvol, double* dL_dPhat, double* dL_dproj) {
  const size_t img = (size_t)nu * nv;
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < V; ++j) {
    const double* M = Phat + 12 * j;
    const double* d = proj + img * j;
    double* gu = NULL;
    double* gv = NULL;
    if (dL_dPhat && deriv_mode == ORC_DERIV_CENTRAL) {
      gu = (double*)malloc(img * sizeof(double));
      gv = (double*)malloc(img * sizeof(double));
      orc_gradient_images(d, nu, nv, gu, gv);
    }
    double G[12] = {0};
    double* dd = dL_dproj ? dL_dproj + img * j : NULL;
    if (dd) memset(dd, 0, img * sizeof(double));
    double c = view_weight ? view_weight[j] : 1.0;
    for (int k = 0; k < g->nz; ++k)
      for (int jy = 0; jy < g->ny; ++jy)
        for (int i = 0; i < g->nx; ++i) {
          double delta = dL_dvol[((size_t)k * g->ny + jy) * g->nx + i];
          double p[4];
          voxel_pos(g, i, jy, k, p);
          double u = M[0] * p[0] + M[1] * p[1] + M[2] * p[2] + M[3];
          double v = M[4] * p[0] + M[5] * p[1] + M[6] * p[2] + M[7];
          double w = M[8] * p[0] + M[9] * p[1] + M[10] * p[2] + M[11];
          if (!(w > 0.0)) continue;
          double ub = u / w, vb = v / w;
          orc_loc L = locate(ub, vb, nu, nv);
          if (!L.inside) continue;
          double om = (weight_mode == ORC_WEIGHT_FDK) ? (sid / w) * (sid / w) : 1.0;
          double s = delta * c * om;
          if (dL_dPhat) {
            double g_u, g_v;
            if (deriv_mode == ORC_DERIV_CENTRAL) {
              g_u = bilerp(gu, nu, nv, L);
              g_v = bilerp(gv, nu, nv, L);
            } else {
              double d00 = tap(d, nu, nv, L.iu, L.iv), d10 = tap(d, nu, nv, L.iu + 1, L.iv);
              double d01 = tap(d, nu, nv, L.iu, L.iv + 1), d11 = tap(d, nu, nv, L.iu + 1, L.iv + 1);
              g_u = (1 - L.fv) * (d10 - d00) + L.fv * (d11 - d01);
              g_v = (1 - L.fu) * (d01 - d00) + L.fu * (d11 - d10);
            }
            /* Eq. 4: rows g_u p~/w, g_v p~/w, -h(p~)/w^2 with h from Eq. 5,
             * h(i) = (g_u u + g_v v) i, u and v homogeneous. */
            double a0 = s * g_u / w;
            double a1 = s * g_v / w;
            double a2 = -s * (g_u * u + g_v * v) / (w * w);
            if (weight_mode == ORC_WEIGHT_FDK) {
              double val = bilerp(d, nu, nv, L);
              a2 += delta * c * val * (-2.0 * om / w); /* d omega / d w */
            }
            for (int q = 0; q < 4; ++q) {
              G[q] += a0 * p[q];
              G[4 + q] += a1 * p[q];
              G[8 + q] += a2 * p[q];
            }
          }
          if (dd) {
            double wts[4] = {(1 - L.fu) * (1 - L.fv), L.fu * (1 - L.fv), (1 - L.fu) * L.fv,
                             L.fu * L.fv};
            long as[4] = {L.iu, L.iu + 1, L.iu, L.iu + 1};
            long bs[4] = {L.iv, L.iv, L.iv + 1, L.iv + 1};
            for (int t = 0; t < 4; ++t)
              if (as[t] >= 0 && bs[t] >= 0 && as[t] < nu && bs[t] < nv)
                dd[(size_t)bs[t] * nu + (size_t)as[t]] += s * wts[t];
          }
        }
    if (dL_dPhat) memcpy(dL_dPhat + 12 * j, G, sizeof G);
    free(gu);
    free(gv);
  }
}

/* Chain rule (Eq. 2) through Eq. 1:
 *   dL/dtheta_{j,m} = < dL/dPhat_j , P_j dT/dtheta_m(theta_j) >_F. */
void orc_chain_motion(int V, const double* P, const double* theta, const double* dL_dPhat,
                      double* dL_dtheta) {
  for (int j = 0; j < V; ++j) {
    double dT[96];
    orc_rigid_grad(theta + 6 * j, dT);
    for (int m = 0; m < 6; ++m) {
      double J[12];
      mat34_mul44(P + 12 * j, dT + 16 * m, J);
      double s = 0.0;
      for (int e = 0; e < 12; ++e) s += dL_dPhat[12 * j + e] * J[e];
      dL_dtheta[6 * j + m] = s;
    }
  }
}

/* ---------------------------------------------------- loss and optimizers */

/* Sharpness loss: L = -(1/K) sum over the three axes of the squared forward
 * differences over all voxel pairs inside the volume, K = nx*ny*nz; grad
 * receives dL/dI.  Returns L. */
double orc_sharpness(const orc_vol* g, const double* vol, double* grad) {
  const long nx = g->nx, ny = g->ny, nz = g->nz;
  const double K = (double)nx * ny * nz;
  double L = 0.0;
  if (grad) memset(grad, 0, sizeof(double) * nx * ny * nz);
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        size_t x = ((size_t)k * ny + j) * nx + i;
        long nb[3][4] = {{i + 1, j, k, 1}, {i, j + 1, k, nx}, {i, j, k + 1, nx * ny}};
        for (int a = 0; a < 3; ++a) {
          if (nb[a][0] >= nx || nb[a][1] >= ny || nb[a][2] >= nz) continue;
          size_t y = x + (size_t)nb[a][3];
          double diff = vol[y] - vol[x];
          L -= diff * diff / K;
          if (grad) {
            grad[y] -= 2.0 * diff / K;
            grad[x] += 2.0 * diff / K;
          }
        }
      }
  return L;
}

/* Total variation (isotropic, smoothed), the classical autofocus metric the
 * paper compares against (Sec. IV-A):
 *   L = (1/K) sum over voxels x with all three forward neighbours inside of
 *       sqrt(|grad+ I(x)|^2 + eps^2),  grad+ = forward differences,
 * K = nx*ny*nz; grad receives dL/dI.  Returns L. */
double orc_tv(const orc_vol* g, const double* vol, double eps, double* grad) {
  const long nx = g->nx, ny = g->ny, nz = g->nz;
  const double K = (double)nx * ny * nz;
  double L = 0.0;
  if (grad) memset(grad, 0, sizeof(double) * nx * ny * nz);
  for (long k = 0; k + 1 < nz; ++k)
    for (long j = 0; j + 1 < ny; ++j)
      for (long i = 0; i + 1 < nx; ++i) {
        size_t x = ((size_t)k * ny + j) * nx + i;
        double gx = vol[x + 1] - vol[x];
        double gy = vol[x + nx] - vol[x];
        double gz = vol[x + (size_t)nx * ny] - vol[x];
        double n = sqrt(gx * gx + gy * gy + gz * gz + eps * eps);
        L += n / K;
        if (grad) {
          grad[x + 1] += gx / n / K;
          grad[x + nx] += gy / n / K;
          grad[x + (size_t)nx * ny] += gz / n / K;
          grad[x] -= (gx + gy + gz) / n / K;
        }
      }
  return L;
}

/* Remove the per-parameter mean over views (gauge of a global rigid motion). */
static void remove_mean(int V, double* theta) {
  for (int m = 0; m < 6; ++m) {
    double s = 0.0;
    for (int j = 0; j < V; ++j) s += theta[6 * j + m];
    s /= V;
    for (int j = 0; j < V; ++j) theta[6 * j + m] -= s;
  }
}

/* Eq. 6: x <- x - s0 t^n df/dx, then the gauge step. */
void orc_gd_step(int V, double* theta, const double* grad, double s0, double t, int n,
                 int gauge) {
  double step = s0 * pow(t, n);
  for (int e = 0; e < 6 * V; ++e) theta[e] -= step * grad[e];
  if (gauge) remove_mean(V, theta);
}

/* Adam (Kingma & Ba), iteration counter n starting at 1, then the gauge step. */
void orc_adam_step(int V, double* theta, const double* grad, double* m1, double* m2, double lr,
                   double b1, double b2, double eps, int n, int gauge) {
  double c1 = 1.0 - pow(b1, n), c2 = 1.0 - pow(b2, n);
  for (int e = 0; e < 6 * V; ++e) {
    m1[e] = b1 * m1[e] + (1.0 - b1) * grad[e];
    m2[e] = b2 * m2[e] + (1.0 - b2) * grad[e] * grad[e];
    double mh = m1[e] / c1, vh = m2[e] / c2;
    theta[e] -= lr * mh / (sqrt(vh) + eps);
  }
  if (gauge) remove_mean(V, theta);
}

/* ------------------------------------------------------------------ RPE */

/* Reprojection error: mean detector distance in mm (pixel distance scaled by
 * the pixel pitch du, dv) between the projections of npts world points under
 * Pa_j and Pb_j, over all points and views. */
double orc_rpe(int V, const double* Pa, const double* Pb, int npts, const double* pts, double du,
               double dv) {
  double s = 0.0;
  for (int j = 0; j < V; ++j)
    for (int q = 0; q < npts; ++q) {
      const double* x = pts + 3 * q;
      double ua[3], ub[3];
      for (int r = 0; r < 3; ++r) {
        ua[r] = Pa[12 * j + 4 * r] * x[0] + Pa[12 * j + 4 * r + 1] * x[1] +
                Pa[12 * j + 4 * r + 2] * x[2] + Pa[12 * j + 4 * r + 3];
        ub[r] = Pb[12 * j + 4 * r] * x[0] + Pb[12 * j + 4 * r + 1] * x[1] +
                Pb[12 * j + 4 * r + 2] * x[2] + Pb[12 * j + 4 * r + 3];
      }
      double du_ = (ua[0] / ua[2] - ub[0] / ub[2]) * du;
      double dv_ = (ua[1] / ua[2] - ub[1] / ub[2]) * dv;
      s += sqrt(du_ * du_ + dv_ * dv_);
    }
  return s / ((double)V * npts);
}

int orc_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Akima spline motion model (Sec. II-B.1): each of the six motion
 * parameters is an Akima spline through N_n node values at knots spread
 * evenly over the scan, first knot at the first view and last knot at the
 * last; theta_j is the splines evaluated at view j's time.
 *
 * Akima's construction, in the order it is defined:
 *   secants      m_i = (y_{i+1} - y_i) / (x_{i+1} - x_i),     i = 0 .. n-2
 *   end secants  two more at each end by linear extrapolation of the
 *                secant sequence: m_{-1} = 2 m_0 - m_1, m_{-2} = 2 m_{-1} - m_0,
 *                m_{n-1} = 2 m_{n-2} - m_{n-3}, m_n = 2 m_{n-1} - m_{n-2}
 *   node slopes  t_i = (|m_{i+1} - m_i| m_{i-1} + |m_{i-1} - m_{i-2}| m_i)
 *                      / (|m_{i+1} - m_i| + |m_{i-1} - m_{i-2}|),
 *                and (m_{i-1} + m_i) / 2 where the denominator is 0
 *   pieces       the cubic Hermite interpolant of (y_i, t_i), (y_{i+1}, t_{i+1})
 *                on [x_i, x_{i+1}].
 * Needs n >= 3.
 *
 * Every quantity is carried as a dual number (value, derivative along one
 * direction dy of the node values), so one pass also gives one column of
 * the Jacobian d(spline values)/d(node values): forward-mode
 * differentiation written out, independent of any reverse-mode code.
 * ---------------------------------------------------------------------- */
typedef struct { double v, d; } orc_dual;

static orc_dual dl_add(orc_dual a, orc_dual b) { orc_dual r = {a.v + b.v, a.d + b.d}; return r; }
static orc_dual dl_sub(orc_dual a, orc_dual b) { orc_dual r = {a.v - b.v, a.d - b.d}; return r; }
static orc_dual dl_scale(double s, orc_dual a) { orc_dual r = {s * a.v, s * a.d}; return r; }
static orc_dual dl_mul(orc_dual a, orc_dual b) {
  orc_dual r = {a.v * b.v, a.d * b.v + a.v * b.d};
  return r;
}
static orc_dual dl_div(orc_dual a, orc_dual b) {
  orc_dual r = {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)};
  return r;
}
static orc_dual dl_abs(orc_dual a) {
  const double s = a.v > 0.0 ? 1.0 : (a.v < 0.0 ? -1.0 : 0.0);
  orc_dual r = {fabs(a.v), s * a.d};
  return r;
}

/* Values (and derivatives along dy, which may be NULL for zero) of the
 * spline through (x_i, y_i), i < n, at the m points xe; n >= 3. */
static void akima_dual(int n, const double* x, const double* y, const double* dy, int m,
                       const double* xe, double* out, double* dout) {
  orc_dual* s = (orc_dual*)malloc(sizeof(orc_dual) * (size_t)(n + 3)); /* s[k] = m_{k-2} */
  orc_dual* t = (orc_dual*)malloc(sizeof(orc_dual) * (size_t)n);
  for (int i = 0; i + 1 < n; ++i) {
    const orc_dual a = {y[i], dy ? dy[i] : 0.0}, b = {y[i + 1], dy ? dy[i + 1] : 0.0};
    s[i + 2] = dl_scale(1.0 / (x[i + 1] - x[i]), dl_sub(b, a));
  }
  s[1] = dl_sub(dl_scale(2.0, s[2]), s[3]);
  s[0] = dl_sub(dl_scale(2.0, s[1]), s[2]);
  s[n + 1] = dl_sub(dl_scale(2.0, s[n]), s[n - 1]);
  s[n + 2] = dl_sub(dl_scale(2.0, s[n + 1]), s[n]);
  for (int i = 0; i < n; ++i) {
    /* m_{i-2} = s[i], m_{i-1} = s[i+1], m_i = s[i+2], m_{i+1} = s[i+3] */
    const orc_dual w1 = dl_abs(dl_sub(s[i + 3], s[i + 2]));
    const orc_dual w2 = dl_abs(dl_sub(s[i + 1], s[i]));
    const orc_dual den = dl_add(w1, w2);
    if (den.v == 0.0)
      t[i] = dl_scale(0.5, dl_add(s[i + 1], s[i + 2]));
    else
      t[i] = dl_div(dl_add(dl_mul(w1, s[i + 1]), dl_mul(w2, s[i + 2])), den);
  }
  for (int q = 0; q < m; ++q) {
    int i = 0;
    while (i < n - 2 && xe[q] >= x[i + 1]) ++i;
    const double h = x[i + 1] - x[i], e = xe[q] - x[i];
    const orc_dual yi = {y[i], dy ? dy[i] : 0.0};
    const orc_dual mi = s[i + 2];
    /* p = y_i + t_i e + c e^2 + d e^3 with c = (3 m_i - 2 t_i - t_{i+1}) / h,
       d = (t_i + t_{i+1} - 2 m_i) / h^2 */
    const orc_dual c = dl_scale(1.0 / h, dl_sub(dl_sub(dl_scale(3.0, mi), dl_scale(2.0, t[i])), t[i + 1]));
    const orc_dual d = dl_scale(1.0 / (h * h), dl_sub(dl_add(t[i], t[i + 1]), dl_scale(2.0, mi)));
    const orc_dual p = dl_add(dl_add(yi, dl_scale(e, t[i])), dl_add(dl_scale(e * e, c), dl_scale(e * e * e, d)));
    out[q] = p.v;
    if (dout) dout[q] = p.d;
  }
  free(s);
  free(t);
}

/* Spline values at xe (m points) through n >= 3 knots (x, y). */
void orc_akima_eval(int n, const double* x, const double* y, int m, const double* xe, double* out) {
  akima_dual(n, x, y, NULL, m, xe, out, NULL);
}

/* Jacobian J[q][k] = d spline(xe_q) / d y_k, m x n, by forward-mode duals. */
void orc_akima_jacobian(int n, const double* x, const double* y, int m, const double* xe,
                        double* J) {
  double* dy = (double*)calloc((size_t)n, sizeof(double));
  double* out = (double*)malloc(sizeof(double) * (size_t)m);
  double* dout = (double*)malloc(sizeof(double) * (size_t)m);
  for (int k = 0; k < n; ++k) {
    dy[k] = 1.0;
    akima_dual(n, x, y, dy, m, xe, out, dout);
    for (int q = 0; q < m; ++q) J[(size_t)q * n + k] = dout[q];
    dy[k] = 0.0;
  }
  free(dy);
  free(out);
  free(dout);
}

/* ------------------------------------------------------------------------
 * FDK preprocessing of the raw line integrals (Sec. III: "a ramp filter and a
 * cosine filter are applied to the computed projection images"; short-scan
 * redundancy weights for the 200-degree arcs), written as its definition:
 *   q[j][b][a] = tau * sum_k h[a - k] * w_j(k) * c(k, b) * p[j][b][k],
 *   c(a, b)   = SDD / sqrt(SDD^2 + x_a^2 + y_b^2)  (cosine weight; x_a, y_b in
 *               mm from the principal point (nu-1)/2, (nv-1)/2),
 *   h[n]      = -2 / (pi^2 tau^2 (4 n^2 - 1))      (Shepp-Logan ramp),
 *   tau       = pitch * SID / SDD                 (detector scaled to the isocenter),
 *   w_j(k)    = Parker's short-scan weight of view j at fan angle
 *               gamma = atan(x_k / SDD), generalised to over-scan by using
 *               delta = (arc - pi)/2 for the maximum fan angle; 1/2 for a full
 *               scan (arc >= 2 pi, every ray measured twice).
 * Views are spread as in the geometry: beta_j - beta_0 = j * arc / (V - 1)
 * for short scans.  A plain O(nu^2) convolution per row.
 * ---------------------------------------------------------------------- */
double orc_parker(double beta, double gamma, double arc) {
  const double pi = 3.14159265358979323846;
  const double delta = 0.5 * (arc - pi);
  double w;
  if (beta < 2.0 * delta + 2.0 * gamma) {
    const double s = sin(0.25 * pi * beta / (delta + gamma));
    w = s * s;
  } else if (beta > pi + 2.0 * gamma) {
    const double s = sin(0.25 * pi * (pi + 2.0 * delta - beta) / (delta - gamma));
    w = s * s;
  } else {
    w = 1.0;
  }
  return w < 0.0 ? 0.0 : (w > 1.0 ? 1.0 : w);
}

void orc_fdk_filter(int V, int nu, int nv, const double* raw, double pitch, double sid, double sdd,
                    double arc, int ext, double* out) {
  /* ext > 0: truncation correction (Sec. IV-D) -- each weighted row is
     extended by ext pixels on either side, falling linearly from its edge
     value to 0 (the value at extension pixel m = 1..ext is edge * (1 - m/ext)),
     filtered, and the measured nu pixels are kept. */
  const double pi = 3.14159265358979323846;
  const double tau = pitch * sid / sdd;
  const int full = arc >= 2.0 * pi - 1e-12;
  const double dbeta = full ? arc / V : (V > 1 ? arc / (V - 1) : 0.0);
  const int n = nu + 2 * ext;                                          /* extended row */
  double* h = (double*)malloc(sizeof(double) * (size_t)(2 * n - 1)); /* h[m + n - 1] */
  for (int m = -(n - 1); m <= n - 1; ++m)
    h[m + n - 1] = -2.0 / (pi * pi * tau * tau * (4.0 * (double)m * m - 1.0));
#pragma omp parallel for schedule(static)
  for (int j = 0; j < V; ++j) {
    double* row = (double*)malloc(sizeof(double) * (size_t)n);
    const double beta = j * dbeta;
    for (int b = 0; b < nv; ++b) {
      const double y = (b - 0.5 * (nv - 1)) * pitch;
      for (int k = 0; k < nu; ++k) {
        const double x = (k - 0.5 * (nu - 1)) * pitch;
        const double c = sdd / sqrt(sdd * sdd + x * x + y * y);
        const double w = full ? 0.5 : orc_parker(beta, atan(x / sdd), arc);
        row[k + ext] = w * c * raw[((size_t)j * nv + b) * nu + k];
      }
      for (int m = 1; m <= ext; ++m) {
        row[ext - m] = row[ext] * (1.0 - (double)m / ext);
        row[ext + nu - 1 + m] = row[ext + nu - 1] * (1.0 - (double)m / ext);
      }
      for (int a = 0; a < nu; ++a) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += h[(a + ext) - k + n - 1] * row[k];
        out[((size_t)j * nv + b) * nu + a] = tau * s;
      }
    }
    free(row);
  }
  free(h);
}

/* Threads of the OpenMP loops from now on (1 = single-threaded timing). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  extern void omp_set_num_threads(int);
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}
