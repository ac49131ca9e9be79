/*
 * FP64 oracle for X-Gaussian's Differentiable Radiative Rasterization (arXiv 2403.04116).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline call this file.  It shares no code, header, helper or constant table with the
 * CUDA library and it never calls it.
 *
 * What it computes, pixel by pixel and with no tiles:
 *   - camera from the scanner parameters (Sec. 3.3, Eq. 12): M_ext rows (-sin p, cos p, 0 | 0),
 *     (0, 0, -1 | 0), (-cos p, -sin p, 0 | L_SO); M_int with focal L_SD and principal point
 *     (W/2, H/2).  The focal is taken in pixels, L_SD / pitch (the paper uses pitch 1 mm).
 *   - Sigma = R S S^T R^T from a quaternion (w, x, y, z) normalised here and a scale vector
 *     (Sec. 3.1, Eq. 1 text).
 *   - t = M_ext mu, u = M_int t (Eq. 7); Sigma' = J W Sigma W^T J^T with J, W of Eq. 9
 *     (Eq. 8); Sigma'' = its top-left 2x2 block (Sec. 3.2) plus 0.3 px^2 on the diagonal.
 *   - for pixel p the 2-D density exp(-1/2 d^T Sigma''^-1 d), d = u - p, p the pixel centre
 *     (x + 1/2, y + 1/2); sigma = min(0.99, opacity * density); Gaussians with t_z <= near,
 *     det Sigma'' <= 0 or sigma < 1/255 are left out; the rest are ordered by ascending t_z
 *     (ties: ascending index) and blended front to back, I(p) = sum_j i_j sigma_j prod_{k<j}
 *     (1 - sigma_k) (Eq. 10), stopping before the first Gaussian that would take the
 *     transmittance below 1e-4; background 0.
 *   - gradients of L = sum_p G(p) I(p) for a given G: the per-pixel reverse recursion of
 *     Eq. 10 (transmittance stored on the way forward), then the chain rule back through
 *     Eq. 9, 8, 7 and Sigma = R S S^T R^T to mean, scale, quaternion, opacity, intensity.
 *
 * The Gaussian-pixel cost is brute force.  The only acceleration is a bounding-box
 * prefilter that cannot drop an included Gaussian, nor one within the ambiguity margin of
 * the inclusion threshold: sigma >= (1 - m)/255 needs |d|^2 <= 2 ln(255 o / (1 - m))
 * lambda_max(Sigma''), and the box is that radius with a margin.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  double sod, sdd, pitch_u, pitch_v, angle;
  int32_t width, height;
} xo_view;

typedef struct {
  int ok;
  double W[3][3];          /* viewing rotation (Eq. 9) */
  double t[3];             /* camera coordinates (Eq. 7) */
  double u[2];             /* detector coordinates (Eq. 7) */
  double J[3][3];          /* Eq. 9 */
  double Sigma[3][3];      /* world covariance */
  double R[3][3], s[3], qn[4], qnorm;
  double cov[3];           /* Sigma'' entries (A, B, C) incl. dilation */
  double K[3];             /* conic (a, b, c) = inverse of Sigma'' */
  double o, i;
  double bx0, bx1, by0, by1; /* prefilter box on pixel-centre coordinates */
} xo_pg;

#define XO_DILATE 0.3
#define XO_ALPHA_MIN (1.0 / 255.0)
#define XO_ALPHA_MAX 0.99
#define XO_T_MIN 1e-4

/* decision margins for the ambiguity flags (relative) */
#define XO_MARGIN_ALPHA 1e-4
#define XO_MARGIN_T 1e-3
#define XO_MARGIN_DEPTH (1.0 / 4194304.0) /* 2^-22: two float32 ulps of t_z */

static void mat3_mul(const double A[3][3], const double B[3][3], double C[3][3]) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[r][k] * B[k][c];
      C[r][c] = s;
    }
}

static void mat3_transpose(const double A[3][3], double At[3][3]) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) At[r][c] = A[c][r];
}

/* rotation of the unit quaternion q = (w, x, y, z) */
static void quat_rot(const double q[4], double R[3][3]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1.0 - 2.0 * (y * y + z * z);
  R[0][1] = 2.0 * (x * y - w * z);
  R[0][2] = 2.0 * (x * z + w * y);
  R[1][0] = 2.0 * (x * y + w * z);
  R[1][1] = 1.0 - 2.0 * (x * x + z * z);
  R[1][2] = 2.0 * (y * z - w * x);
  R[2][0] = 2.0 * (x * z - w * y);
  R[2][1] = 2.0 * (y * z + w * x);
  R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

/* dR/dq_k for the unit quaternion, k = w, x, y, z */
static void quat_rot_deriv(const double q[4], double D[4][3][3]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double dw[3][3] = {{0, -2 * z, 2 * y}, {2 * z, 0, -2 * x}, {-2 * y, 2 * x, 0}};
  double dx[3][3] = {{0, 2 * y, 2 * z}, {2 * y, -4 * x, -2 * w}, {2 * z, 2 * w, -4 * x}};
  double dy[3][3] = {{-4 * y, 2 * x, 2 * w}, {2 * x, 0, 2 * z}, {-2 * w, 2 * z, -4 * y}};
  double dz[3][3] = {{-4 * z, -2 * w, 2 * x}, {2 * w, -4 * z, 2 * y}, {2 * x, 2 * y, 0}};
  memcpy(D[0], dw, sizeof dw);
  memcpy(D[1], dx, sizeof dx);
  memcpy(D[2], dy, sizeof dy);
  memcpy(D[3], dz, sizeof dz);
}

static void view_matrices(const xo_view* v, double W[3][3], double* L, double* fu, double* fv) {
  double s = sin(v->angle), c = cos(v->angle);
  double Wm[3][3] = {{-s, c, 0.0}, {0.0, 0.0, -1.0}, {-c, -s, 0.0}};
  memcpy(W, Wm, sizeof Wm);
  *L = v->sod;
  *fu = v->sdd / v->pitch_u;
  *fv = v->sdd / v->pitch_v;
}

/* Project Gaussian g under view v (Eq. 7-9 and the Sigma'' block). */
static void project_one(int64_t n, int64_t g, const double* mean, const double* scale, const double* quat,
                        const double* opac, const double* inten, const xo_view* v, double near_mm,
                        xo_pg* pg) {
  memset(pg, 0, sizeof *pg);
  double mu[3] = {mean[g], mean[n + g], mean[2 * n + g]};
  double q[4] = {quat[g], quat[n + g], quat[2 * n + g], quat[3 * n + g]};
  double s[3] = {scale[g], scale[n + g], scale[2 * n + g]};
  double o = opac[g], in = inten[g];
  for (int k = 0; k < 3; ++k)
    if (!isfinite(mu[k]) || !isfinite(s[k])) return;
  for (int k = 0; k < 4; ++k)
    if (!isfinite(q[k])) return;
  if (!isfinite(o) || !isfinite(in)) return;
  double qq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(qq > 0.0)) return;
  for (int k = 0; k < 4; ++k) pg->qn[k] = q[k] / qq;
  pg->qnorm = qq;
  quat_rot(pg->qn, pg->R);
  double M[3][3], Mt[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) M[r][c] = pg->R[r][c] * s[c];
  mat3_transpose(M, Mt);
  mat3_mul(M, Mt, pg->Sigma);
  for (int k = 0; k < 3; ++k) pg->s[k] = s[k];

  double L, fu, fv;
  view_matrices(v, pg->W, &L, &fu, &fv);
  for (int r = 0; r < 3; ++r) pg->t[r] = pg->W[r][0] * mu[0] + pg->W[r][1] * mu[1] + pg->W[r][2] * mu[2];
  pg->t[2] += L;
  double tx = pg->t[0], ty = pg->t[1], tz = pg->t[2];
  if (!(tz > near_mm)) return;
  pg->u[0] = fu * tx / tz + 0.5 * v->width;
  pg->u[1] = fv * ty / tz + 0.5 * v->height;
  double J[3][3] = {{fu / tz, 0.0, -fu * tx / (tz * tz)}, {0.0, fv / tz, -fv * ty / (tz * tz)}, {0.0, 0.0, 0.0}};
  memcpy(pg->J, J, sizeof J);
  double P[3][3], Pt[3][3], PS[3][3], Sp[3][3];
  mat3_mul(J, pg->W, P);
  mat3_transpose(P, Pt);
  mat3_mul(P, pg->Sigma, PS);
  mat3_mul(PS, Pt, Sp);
  double A = Sp[0][0] + XO_DILATE, B = Sp[0][1], C = Sp[1][1] + XO_DILATE;
  double det = A * C - B * B;
  if (!(det > 0.0)) return;
  pg->cov[0] = A;
  pg->cov[1] = B;
  pg->cov[2] = C;
  pg->K[0] = C / det;
  pg->K[1] = -B / det;
  pg->K[2] = A / det;
  pg->o = o;
  pg->i = in;
  /* Candidates are the Gaussians whose sigma can reach the inclusion threshold or come
   * within the ambiguity margin below it: those below the threshold are never blended,
   * but a pixel where one sits within the margin is flagged. */
  if (!(o * 255.0 >= 1.0 - XO_MARGIN_ALPHA)) return;
  double mid = 0.5 * (A + C);
  double lam = mid + sqrt(fmax(mid * mid - det, 0.0));
  double r = sqrt(2.0 * log(255.0 * o / (1.0 - XO_MARGIN_ALPHA)) * lam) * (1.0 + 1e-9) + 1e-9;
  if (!isfinite(r) || !isfinite(pg->u[0]) || !isfinite(pg->u[1])) return;
  pg->bx0 = pg->u[0] - r;
  pg->bx1 = pg->u[0] + r;
  pg->by0 = pg->u[1] - r;
  pg->by1 = pg->u[1] + r;
  pg->ok = 1;
}

/* ----------------------------------------------------------------------------------- */

typedef struct {
  double tz;
  int64_t id;
  double alpha;  /* min(0.99, o e^power) */
  double a0;     /* o e^power before the clamp */
  double e;      /* e^power */
  double dx, dy; /* u - p */
  int pass;      /* a0 >= 1/255 */
  int near_thr;  /* a0 within the margin of 1/255 */
} xo_cand;

static int cand_cmp(const void* pa, const void* pb) {
  const xo_cand* a = (const xo_cand*)pa;
  const xo_cand* b = (const xo_cand*)pb;
  if (a->tz < b->tz) return -1;
  if (a->tz > b->tz) return 1;
  return (a->id < b->id) ? -1 : (a->id > b->id);
}

typedef struct {
  int64_t* start; /* [H + 1] */
  int64_t* ids;
} xo_rows;

static int build_rows(int64_t n, const xo_pg* pg, int H, xo_rows* rows) {
  rows->start = (int64_t*)calloc((size_t)H + 1, sizeof(int64_t));
  if (!rows->start) return -1;
  for (int64_t g = 0; g < n; ++g) {
    if (!pg[g].ok) continue;
    int y0 = (int)fmax(ceil(pg[g].by0 - 0.5), 0.0);
    int y1 = (int)fmin(floor(pg[g].by1 - 0.5), (double)(H - 1));
    for (int y = y0; y <= y1; ++y) rows->start[y + 1]++;
  }
  for (int y = 0; y < H; ++y) rows->start[y + 1] += rows->start[y];
  rows->ids = (int64_t*)malloc(sizeof(int64_t) * (size_t)(rows->start[H] > 0 ? rows->start[H] : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)H);
  if (!rows->ids || !fill) return -1;
  memcpy(fill, rows->start, sizeof(int64_t) * (size_t)H);
  for (int64_t g = 0; g < n; ++g) {
    if (!pg[g].ok) continue;
    int y0 = (int)fmax(ceil(pg[g].by0 - 0.5), 0.0);
    int y1 = (int)fmin(floor(pg[g].by1 - 0.5), (double)(H - 1));
    for (int y = y0; y <= y1; ++y) rows->ids[fill[y]++] = g;
  }
  free(fill);
  return 0;
}

static void free_rows(xo_rows* rows) {
  free(rows->start);
  free(rows->ids);
}

/* Candidates of pixel (x, y), sorted by (t_z, index).  Returns their count. */
static int64_t gather(const xo_pg* pg, const xo_rows* rows, int x, int y, xo_cand* out) {
  double px = x + 0.5, py = y + 0.5;
  int64_t m = 0;
  for (int64_t k = rows->start[y]; k < rows->start[y + 1]; ++k) {
    int64_t g = rows->ids[k];
    const xo_pg* p = &pg[g];
    if (px < p->bx0 || px > p->bx1) continue;
    double dx = p->u[0] - px, dy = p->u[1] - py;
    double power = -0.5 * (p->K[0] * dx * dx + 2.0 * p->K[1] * dx * dy + p->K[2] * dy * dy);
    double e = exp(power);
    double a0 = p->o * e;
    int pass = a0 >= XO_ALPHA_MIN;
    int near_thr = fabs(a0 * 255.0 - 1.0) < XO_MARGIN_ALPHA;
    if (!pass && !near_thr) continue;
    xo_cand c;
    c.tz = p->t[2];
    c.id = g;
    c.a0 = a0;
    c.alpha = a0 < XO_ALPHA_MAX ? a0 : XO_ALPHA_MAX;
    c.e = e;
    c.dx = dx;
    c.dy = dy;
    c.pass = pass;
    c.near_thr = near_thr;
    out[m++] = c;
  }
  qsort(out, (size_t)m, sizeof(xo_cand), cand_cmp);
  return m;
}

/* Blend the sorted candidates (Eq. 10).  Writes the contributors' positions in `cand` to
 * `contrib` and their transmittance before blending to `Tb`.  Returns the count. */
static int64_t blend(const xo_pg* pg, const xo_cand* cand, int64_t m, double* C_out, double* T_out,
                     int64_t* contrib, double* Tb, uint8_t* amb) {
  double T = 1.0, C = 0.0;
  int64_t n = 0;
  uint8_t flags = 0;
  double prev_tz = -1.0;
  for (int64_t k = 0; k < m; ++k) {
    const xo_cand* c = &cand[k];
    if (c->near_thr) flags |= 1;
    if (!c->pass) continue;
    if (prev_tz > 0.0 && fabs(c->tz - prev_tz) <= XO_MARGIN_DEPTH * c->tz) flags |= 4;
    prev_tz = c->tz;
    double Tn = T * (1.0 - c->alpha);
    if (fabs(Tn / XO_T_MIN - 1.0) < XO_MARGIN_T) flags |= 2;
    if (Tn < XO_T_MIN) {
      /* The candidates after the one that stops the blend are left out, but one within
       * rounding of its depth may come before it in a float32 depth order (and be blended
       * in its place): that order is ambiguous too. */
      for (int64_t q = k + 1; q < m; ++q) {
        if (!cand[q].pass && !cand[q].near_thr) continue;
        if (fabs(cand[q].tz - c->tz) <= XO_MARGIN_DEPTH * cand[q].tz) flags |= 4;
        break;
      }
      break;
    }
    if (contrib) contrib[n] = k;
    if (Tb) Tb[n] = T;
    C += pg[c->id].i * c->alpha * T;
    T = Tn;
    ++n;
  }
  *C_out = C;
  *T_out = T;
  if (amb) *amb = flags;
  return n;
}

static int nthreads_use(int req) {
#ifdef _OPENMP
  return req > 0 ? req : omp_get_max_threads();
#else
  (void)req;
  return 1;
#endif
}

/*
 * Forward image of one view.
 *   mean[3n], scale[3n], quat[4n], opac[n], inten[n]: structure of arrays, activated values.
 *   pix, npix: linear pixel indices y*W + x to evaluate; pix == NULL evaluates all of them.
 *   image, tfinal, ncontrib, amb: W*H arrays; only the evaluated pixels are written.
 * Returns 0, or -1 when memory runs out.
 */
int xo_render(int64_t n, const double* mean, const double* scale, const double* quat, const double* opac,
              const double* inten, const xo_view* view, double near_mm, const int32_t* pix, int64_t npix,
              double* image, double* tfinal, int32_t* ncontrib, uint8_t* amb, int nthreads) {
  int W = view->width, H = view->height;
  xo_pg* pg = (xo_pg*)malloc(sizeof(xo_pg) * (size_t)(n > 0 ? n : 1));
  if (!pg) return -1;
  int nt = nthreads_use(nthreads);
#pragma omp parallel for num_threads(nt) schedule(static)
  for (int64_t g = 0; g < n; ++g) project_one(n, g, mean, scale, quat, opac, inten, view, near_mm, &pg[g]);
  xo_rows rows;
  if (build_rows(n, pg, H, &rows)) {
    free(pg);
    return -1;
  }
  int64_t total = pix ? npix : (int64_t)W * H;
  int err = 0;
#pragma omp parallel num_threads(nt)
  {
    xo_cand* cand = (xo_cand*)malloc(sizeof(xo_cand) * (size_t)(n > 0 ? n : 1));
    if (!cand) {
#pragma omp atomic write
      err = 1;
    }
#pragma omp for schedule(dynamic, 64)
    for (int64_t k = 0; k < total; ++k) {
      if (!cand) continue;
      int64_t p = pix ? pix[k] : k;
      int x = (int)(p % W), y = (int)(p / W);
      int64_t m = gather(pg, &rows, x, y, cand);
      double C, T;
      uint8_t f;
      int64_t nc = blend(pg, cand, m, &C, &T, NULL, NULL, &f);
      image[p] = C;
      if (tfinal) tfinal[p] = T;
      if (ncontrib) ncontrib[p] = (int32_t)nc;
      if (amb) amb[p] = f;
    }
    free(cand);
  }
  free_rows(&rows);
  free(pg);
  return err ? -1 : 0;
}

/* Chain rule of one Gaussian in one view (Eq. 7-9, Sigma = R S S^T R^T): from the 2-D
 * gradients g7 = (dL/du_x, dL/du_y, dL/da, dL/db, dL/dc, dL/do, dL/di) to
 * out12 = (dL/dmean[3], dL/dscale[3], dL/dquat[4], dL/dopacity, dL/dintensity). */
static void chain_rule(const xo_pg* p, const double Wv[3][3], double fu, double fv, const double g7[7],
                       double out12[12]) {
  double gux = g7[0], guy = g7[1], ga = g7[2], gb = g7[3], gc = g7[4];
  /* conic K = S''^-1: dL/dS'' = -K G K with G the symmetric gradient of K
   * (the off-diagonal parameter b sits in two entries, so each gets gb / 2). */
  double Km[2][2] = {{p->K[0], p->K[1]}, {p->K[1], p->K[2]}};
  double Gm[2][2] = {{ga, 0.5 * gb}, {0.5 * gb, gc}};
  double KG[2][2], gS2[2][2];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) KG[r][c] = Km[r][0] * Gm[0][c] + Km[r][1] * Gm[1][c];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) gS2[r][c] = -(KG[r][0] * Km[0][c] + KG[r][1] * Km[1][c]);
  /* Sigma' = P Sigma P^T with P = J W; only its top-left block reaches S''. */
  double gSp[3][3] = {{gS2[0][0], gS2[0][1], 0.0}, {gS2[1][0], gS2[1][1], 0.0}, {0.0, 0.0, 0.0}};
  double P[3][3], Pt[3][3], tmp[3][3], gSigma[3][3], gP[3][3], gJ[3][3], Wt[3][3];
  mat3_mul(p->J, p->W, P);
  mat3_transpose(P, Pt);
  mat3_mul(Pt, gSp, tmp);
  mat3_mul(tmp, P, gSigma);
  mat3_mul(gSp, P, tmp);
  mat3_mul(tmp, p->Sigma, gP);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) gP[r][c] *= 2.0;
  mat3_transpose(p->W, Wt);
  mat3_mul(gP, Wt, gJ);
  double tx = p->t[0], ty = p->t[1], tz = p->t[2];
  double gt[3];
  /* J entries: J00 = fu/tz, J02 = -fu tx/tz^2, J11 = fv/tz, J12 = -fv ty/tz^2 */
  gt[0] = gJ[0][2] * (-fu / (tz * tz));
  gt[1] = gJ[1][2] * (-fv / (tz * tz));
  gt[2] = gJ[0][0] * (-fu / (tz * tz)) + gJ[0][2] * (2.0 * fu * tx / (tz * tz * tz)) +
          gJ[1][1] * (-fv / (tz * tz)) + gJ[1][2] * (2.0 * fv * ty / (tz * tz * tz));
  /* u = (fu tx / tz + W/2, fv ty / tz + H/2) */
  gt[0] += gux * fu / tz;
  gt[1] += guy * fv / tz;
  gt[2] += -gux * fu * tx / (tz * tz) - guy * fv * ty / (tz * tz);
  /* t = W mu + (0, 0, L) */
  for (int c = 0; c < 3; ++c) out12[c] = Wv[0][c] * gt[0] + Wv[1][c] * gt[1] + Wv[2][c] * gt[2];
  /* Sigma = M M^T, M = R S */
  double M[3][3], gM[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) M[r][c] = p->R[r][c] * p->s[c];
  mat3_mul(gSigma, M, gM);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) gM[r][c] *= 2.0;
  double gR[3][3];
  for (int c = 0; c < 3; ++c) {
    double gs = 0.0;
    for (int r = 0; r < 3; ++r) {
      gs += gM[r][c] * p->R[r][c];
      gR[r][c] = gM[r][c] * p->s[c];
    }
    out12[3 + c] = gs;
  }
  double D[4][3][3];
  quat_rot_deriv(p->qn, D);
  double gqn[4];
  for (int k = 0; k < 4; ++k) {
    double a = 0.0;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) a += gR[r][c] * D[k][r][c];
    gqn[k] = a;
  }
  /* qn = q / |q| */
  double dot = 0.0;
  for (int k = 0; k < 4; ++k) dot += gqn[k] * p->qn[k];
  for (int k = 0; k < 4; ++k) out12[6 + k] = (gqn[k] - p->qn[k] * dot) / p->qnorm;
  out12[10] = g7[5];
  out12[11] = g7[6];
}

/*
 * Gradient of L = sum_p G(p) I(p) over the evaluated pixels of one view, ADDED into
 * g_mean[3n], g_scale[3n], g_quat[4n], g_opac[n], g_inten[n] (so calls over several views
 * accumulate).  If g2d is not NULL it receives (overwritten) the per-Gaussian 2-D
 * gradients of this view as 7 planes of n: dL/du_x, dL/du_y, dL/da, dL/db, dL/dc (conic
 * entries, b the off-diagonal), dL/dopacity, dL/dintensity.
 *
 * Magnitudes, for judging floating-point error: if mag2d is not NULL it receives the sum
 * over pixels of |each pixel's term| for the same 7 quantities, and if mag (12 planes of
 * n, the order of the parameter gradients) is not NULL it is ADDED sum_k |A_k| mag2d_k,
 * A_k the parameter gradient that a unit 2-D gradient k produces (the backward pass is
 * linear in the 2-D gradients, so this bounds how term errors reach the parameters).
 */
int xo_render_grad(int64_t n, const double* mean, const double* scale, const double* quat, const double* opac,
                   const double* inten, const xo_view* view, double near_mm, const int32_t* pix, int64_t npix,
                   const double* dL_dimg, double* g_mean, double* g_scale, double* g_quat, double* g_opac,
                   double* g_inten, double* g2d, double* mag2d, double* mag, int nthreads) {
  int W = view->width, H = view->height;
  xo_pg* pg = (xo_pg*)malloc(sizeof(xo_pg) * (size_t)(n > 0 ? n : 1));
  if (!pg) return -1;
  int nt = nthreads_use(nthreads);
#pragma omp parallel for num_threads(nt) schedule(static)
  for (int64_t g = 0; g < n; ++g) project_one(n, g, mean, scale, quat, opac, inten, view, near_mm, &pg[g]);
  xo_rows rows;
  if (build_rows(n, pg, H, &rows)) {
    free(pg);
    return -1;
  }
  const size_t planes = 14; /* 7 sums, 7 sums of magnitudes */
  double* acc = (double*)calloc((size_t)nt * planes * (size_t)n, sizeof(double));
  if (!acc) {
    free_rows(&rows);
    free(pg);
    return -1;
  }
  int64_t total = pix ? npix : (int64_t)W * H;
  int err = 0;
#pragma omp parallel num_threads(nt)
  {
#ifdef _OPENMP
    int tid = omp_get_thread_num();
#else
    int tid = 0;
#endif
    double* my = acc + (size_t)tid * planes * (size_t)n;
    xo_cand* cand = (xo_cand*)malloc(sizeof(xo_cand) * (size_t)(n > 0 ? n : 1));
    int64_t* contrib = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    double* Tb = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!cand || !contrib || !Tb) {
#pragma omp atomic write
      err = 1;
    }
#pragma omp for schedule(dynamic, 64)
    for (int64_t k = 0; k < total; ++k) {
      if (!cand || !contrib || !Tb) continue;
      int64_t p = pix ? pix[k] : k;
      double G = dL_dimg[p];
      if (G == 0.0) continue;
      int x = (int)(p % W), y = (int)(p / W);
      int64_t m = gather(pg, &rows, x, y, cand);
      double C, T;
      int64_t nc = blend(pg, cand, m, &C, &T, contrib, Tb, NULL);
      double A = 0.0; /* intensity carried by everything behind the current contributor */
      for (int64_t j = nc - 1; j >= 0; --j) {
        const xo_cand* c = &cand[contrib[j]];
        int64_t g = c->id;
        double ij = pg[g].i, al = c->alpha, Tj = Tb[j];
        double dC_di = al * Tj;
        double dC_dal = Tj * (ij - A);
        A = al * ij + (1.0 - al) * A;
        double t7[7] = {0, 0, 0, 0, 0, 0, G * dC_di};
        if (c->a0 < XO_ALPHA_MAX) {
          double dL_dal = G * dC_dal;
          t7[5] = dL_dal * c->e;
          double dL_dpow = dL_dal * al;
          const double* K = pg[g].K;
          /* power = -1/2 (a dx^2 + 2 b dx dy + c dy^2), d = u - p */
          t7[0] = dL_dpow * -(K[0] * c->dx + K[1] * c->dy);
          t7[1] = dL_dpow * -(K[1] * c->dx + K[2] * c->dy);
          t7[2] = dL_dpow * -0.5 * c->dx * c->dx;
          t7[3] = dL_dpow * -c->dx * c->dy;
          t7[4] = dL_dpow * -0.5 * c->dy * c->dy;
        }
        for (int q = 0; q < 7; ++q) {
          my[q * n + g] += t7[q];
          my[(7 + q) * n + g] += fabs(t7[q]);
        }
      }
    }
    free(cand);
    free(contrib);
    free(Tb);
  }
  if (err) {
    free(acc);
    free_rows(&rows);
    free(pg);
    return -1;
  }
  for (int t = 1; t < nt; ++t)
    for (size_t k = 0; k < planes * (size_t)n; ++k) acc[k] += acc[(size_t)t * planes * (size_t)n + k];
  if (g2d) memcpy(g2d, acc, sizeof(double) * 7 * (size_t)n);
  if (mag2d) memcpy(mag2d, acc + 7 * (size_t)n, sizeof(double) * 7 * (size_t)n);

  double L, fu, fv, Wv[3][3];
  view_matrices(view, Wv, &L, &fu, &fv);
  double* outs[5] = {g_mean, g_scale, g_quat, g_opac, g_inten};
  const int rows_of[5] = {3, 3, 4, 1, 1};
#pragma omp parallel for num_threads(nt) schedule(static)
  for (int64_t g = 0; g < n; ++g) {
    const xo_pg* p = &pg[g];
    if (!p->ok) continue;
    double g7[7], out12[12];
    for (int q = 0; q < 7; ++q) g7[q] = acc[q * n + g];
    chain_rule(p, Wv, fu, fv, g7, out12);
    int k12 = 0;
    for (int a = 0; a < 5; ++a)
      for (int r = 0; r < rows_of[a]; ++r, ++k12) outs[a][r * n + g] += out12[k12];
    if (mag) {
      double m12[12] = {0};
      for (int q = 0; q < 7; ++q) {
        double e7[7] = {0, 0, 0, 0, 0, 0, 0}, a12[12];
        double mq = acc[(7 + q) * n + g];
        if (mq == 0.0) continue;
        e7[q] = 1.0;
        chain_rule(p, Wv, fu, fv, e7, a12);
        for (int k = 0; k < 12; ++k) m12[k] += fabs(a12[k]) * mq;
      }
      for (int k = 0; k < 12; ++k) mag[k * n + g] += m12[k];
    }
  }
  free(acc);
  free_rows(&rows);
  free(pg);
  return 0;
}

/*
 * Projected quantities of every Gaussian for one view, for pinning the projection step
 * on its own: out[n][12] = ok, t_x, t_y, t_z, u_x, u_y, A, B, C (Sigma'' incl. dilation),
 * a, b, c (conic).
 */
void xo_project(int64_t n, const double* mean, const double* scale, const double* quat, const double* opac,
                const double* inten, const xo_view* view, double near_mm, double* out) {
  for (int64_t g = 0; g < n; ++g) {
    xo_pg p;
    project_one(n, g, mean, scale, quat, opac, inten, view, near_mm, &p);
    double* o = out + 12 * g;
    o[0] = p.ok;
    o[1] = p.t[0];
    o[2] = p.t[1];
    o[3] = p.t[2];
    o[4] = p.u[0];
    o[5] = p.u[1];
    for (int k = 0; k < 3; ++k) {
      o[6 + k] = p.cov[k];
      o[9 + k] = p.K[k];
    }
  }
}
