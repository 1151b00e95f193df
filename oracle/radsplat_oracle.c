/*
 * FP64 CPU oracle for the tile-based Gaussian-splatting hot path of RadSplat
 * (arXiv 2403.13806).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and
 * the CPU-baseline leg of the benchmark call it; the product path never does.
 * It shares no code, header or constant table with the CUDA library.
 *
 * What it states, in the paper's order:
 *   - Sec. 3.2 "Gaussian Splatting": every point has a position p, opacity o,
 *     degree-3 SH coefficients k, scale s and rotation q; Sigma = R S S^T R^T;
 *     the image-space covariance is Sigma' = J M Sigma M^T J^T with M the view
 *     transform and J the Jacobian of the affine approximation of the
 *     perspective projection; alpha_j is the 2D Gaussian times o.
 *   - Eq. (render-gs): c = sum_j c_j alpha_j tau_j with tau_j = prod_{i<j}(1-alpha_i)
 *     over the points sorted front to back.
 *   - Eq. (importance-score): h(p_i) = max over images and rays of alpha_i tau_i.
 *   - Sec. 3.3 pruning mask m_i = 1(h < t_prune); Eq. (importance-score-vis)
 *     visibility mask 1(h > t_cluster); Sec. 3.4 nearest cluster centre.
 * The paper leaves the rasterizer's constants to the 3DGS renderer it cites
 * (Sec. 3.2, Sec. 3.4 "default rasterization"); the readings used here are:
 *   alpha = min(0.99, o * exp(power)); an entry with alpha < 1/255 is skipped
 *   (alpha == 1/255 is kept); an entry with power > 0 is skipped; compositing
 *   stops BEFORE the first entry whose T*(1-alpha) would fall below 1e-4;
 *   Sigma' gets a dilation eps*I; pixel (u,v) samples image point (u,v);
 *   x/z and y/z are clamped to +-1.3 * (half image extent / focal) inside J only;
 *   colour = max(0, 0.5 + sum_lm k_lm Y_lm(d)) with d = normalise(p - camera centre);
 *   the front-to-back order key is the FP32 depth
 *   fmaf(M20,px, fmaf(M21,py, fmaf(M22,pz, m2))), ties broken by the lower index.
 * Everything else is FP64.  The SH basis is built from the associated-Legendre
 * recurrence (real, orthonormal, Condon-Shortley phase, m = -l..l ordering),
 * not from expanded polynomials.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC.  No FMA contraction,
 * so the FP64 arithmetic is exactly what is written here.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_ALPHA_MAX 0.99
#define OR_ALPHA_MIN (1.0 / 255.0)
#define OR_T_MIN 1e-4
#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Spherical harmonics from the associated Legendre recurrence.        */
/* ------------------------------------------------------------------ */

static double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= (double)i;
  return f;
}

/* P_l^m(x) with the Condon-Shortley phase, 0 <= m <= l. */
static double assoc_legendre(int l, int m, double x) {
  double pmm = 1.0;
  double somx2 = sqrt((1.0 - x) * (1.0 + x));
  double fact = 1.0;
  for (int i = 1; i <= m; ++i) {
    pmm = -pmm * fact * somx2;
    fact += 2.0;
  }
  if (l == m) return pmm;
  double pmmp1 = x * (2.0 * m + 1.0) * pmm;
  if (l == m + 1) return pmmp1;
  double pll = 0.0;
  for (int ll = m + 2; ll <= l; ++ll) {
    pll = ((2.0 * ll - 1.0) * x * pmmp1 - (ll + m - 1.0) * pmm) / (ll - m);
    pmm = pmmp1;
    pmmp1 = pll;
  }
  return pll;
}

/* Real orthonormal SH Y_lm for unit direction d, written to y[l*l + l + m]. */
void or_sh_basis(int degree, const double d[3], double* y) {
  double ct = d[2];
  if (ct > 1.0) ct = 1.0;
  if (ct < -1.0) ct = -1.0;
  double phi = atan2(d[1], d[0]);
  for (int l = 0; l <= degree; ++l) {
    for (int m = -l; m <= l; ++m) {
      int am = m < 0 ? -m : m;
      double K = sqrt((2.0 * l + 1.0) / (4.0 * OR_PI) * factorial(l - am) / factorial(l + am));
      double P = assoc_legendre(l, am, ct);
      double v;
      if (m == 0) v = K * P;
      else if (m > 0) v = sqrt(2.0) * K * cos(m * phi) * P;
      else v = sqrt(2.0) * K * sin(am * phi) * P;
      y[l * l + l + m] = v;
    }
  }
}

/* ------------------------------------------------------------------ */
/* Projection (Sec. 3.2): one camera, every Gaussian.                  */
/* ------------------------------------------------------------------ */

static int finite3(const double* v) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

/* Outputs per Gaussian i:
 *   valid[i]   1 if projected (in front of the near plane, finite, det > 0, o >= 1/255)
 *   xy[2i..]   mean2d; conic[3i..] = (a, b, c) of inverse Sigma'; cov2d[3i..] = Sigma'
 *   opacity[i] o; rgb[3i..] colour; depth[i] FP32 order key; ext[2i..] half extents
 *   in pixels of the alpha >= 1/255 ellipse; rect[4i..] tiles (x0, y0, x1, y1),
 *   half-open, covering every pixel of that ellipse's bounding box (empty if none). */
int or_project(int64_t n, const double* means, const double* log_scales, const double* quats,
               const double* logit, const double* sh, int sh_degree, const float* viewmat,
               const float* intr, int width, int height, double eps2d, float near_plane,
               int tile_w, int tile_h, double* xy, double* conic, double* cov2d, double* opacity,
               double* rgb, float* depth, double* ext, int32_t* rect, int32_t* valid) {
  if (sh_degree < 0 || sh_degree > 3) return -1;
  const int ncoef = (sh_degree + 1) * (sh_degree + 1);
  double M[3][3], m[3];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) M[r][c] = viewmat[r * 4 + c];
    m[r] = viewmat[r * 4 + 3];
  }
  /* camera centre = -M^T m */
  double cc[3];
  for (int c = 0; c < 3; ++c) cc[c] = -(M[0][c] * m[0] + M[1][c] * m[1] + M[2][c] * m[2]);
  const double fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3];
  const double lim_x = 1.3 * (0.5 * width / fx);
  const double lim_y = 1.3 * (0.5 * height / fy);
  const int tiles_x = (width + tile_w - 1) / tile_w;
  const int tiles_y = (height + tile_h - 1) / tile_h;

  for (int64_t i = 0; i < n; ++i) {
    valid[i] = 0;
    rect[4 * i + 0] = rect[4 * i + 1] = rect[4 * i + 2] = rect[4 * i + 3] = 0;
    /* the order key is taken in FP32 from the FP32 position (exact for FP32 inputs) */
    const float pxf = (float)means[i], pyf = (float)means[n + i], pzf = (float)means[2 * n + i];
    depth[i] = fmaf(viewmat[8], pxf, fmaf(viewmat[9], pyf, fmaf(viewmat[10], pzf, viewmat[11])));
    double p[3] = {means[i], means[n + i], means[2 * n + i]};
    double ls[3] = {log_scales[i], log_scales[n + i], log_scales[2 * n + i]};
    double q[4] = {quats[i], quats[n + i], quats[2 * n + i], quats[3 * n + i]};
    double lg = logit[i];
    int fin = finite3(p) && finite3(ls) && isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]) &&
              isfinite(q[3]) && isfinite(lg);
    for (int k = 0; k < ncoef * 3 && fin; ++k) fin = isfinite(sh[(int64_t)k * n + i]);
    if (!fin) continue;
    if (!(depth[i] > near_plane)) continue;

    /* rotation from the normalised quaternion (w, x, y, z) */
    double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(qn > 0.0)) continue;
    double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
    double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                      {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                      {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
    double s[3] = {exp(ls[0]), exp(ls[1]), exp(ls[2])};
    /* Sigma = R S S^T R^T */
    double Sig[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
        for (int k = 0; k < 3; ++k) acc += R[r][k] * s[k] * s[k] * R[c][k];
        Sig[r][c] = acc;
      }
    /* t = M p + m */
    double t[3];
    for (int r = 0; r < 3; ++r) t[r] = M[r][0] * p[0] + M[r][1] * p[1] + M[r][2] * p[2] + m[r];
    double tz = t[2];
    double ux = t[0] / tz, uy = t[1] / tz;
    double uxc = ux < -lim_x ? -lim_x : (ux > lim_x ? lim_x : ux);
    double uyc = uy < -lim_y ? -lim_y : (uy > lim_y ? lim_y : uy);
    double J[2][3] = {{fx / tz, 0.0, -fx * uxc / tz}, {0.0, fy / tz, -fy * uyc / tz}};
    /* T = J M (2x3), Sigma' = T Sigma T^T + eps I */
    double T[2][3];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 3; ++c) T[r][c] = J[r][0] * M[0][c] + J[r][1] * M[1][c] + J[r][2] * M[2][c];
    double S2[2][2];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 2; ++c) {
        double acc = 0.0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) acc += T[r][a] * Sig[a][b] * T[c][b];
        S2[r][c] = acc;
      }
    S2[0][0] += eps2d;
    S2[1][1] += eps2d;
    double det = S2[0][0] * S2[1][1] - S2[0][1] * S2[1][0];
    if (!(det > 0.0)) continue;
    double o = 1.0 / (1.0 + exp(-lg));
    if (o < OR_ALPHA_MIN) continue;

    xy[2 * i] = fx * ux + cx;
    xy[2 * i + 1] = fy * uy + cy;
    cov2d[3 * i] = S2[0][0];
    cov2d[3 * i + 1] = S2[0][1];
    cov2d[3 * i + 2] = S2[1][1];
    conic[3 * i] = S2[1][1] / det;
    conic[3 * i + 1] = -S2[0][1] / det;
    conic[3 * i + 2] = S2[0][0] / det;
    opacity[i] = o;

    /* colour from SH along the direction camera centre -> point */
    double d[3] = {p[0] - cc[0], p[1] - cc[1], p[2] - cc[2]};
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    d[0] /= dn;
    d[1] /= dn;
    d[2] /= dn;
    double Y[16];
    or_sh_basis(sh_degree, d, Y);
    for (int ch = 0; ch < 3; ++ch) {
      double acc = 0.5;
      for (int k = 0; k < ncoef; ++k) acc += sh[(int64_t)(k * 3 + ch) * n + i] * Y[k];
      rgb[3 * i + ch] = acc > 0.0 ? acc : 0.0;
    }

    /* support: alpha >= 1/255 <=> d^T conic d <= 2 ln(255 o); bounding box of that ellipse */
    double qq = 2.0 * log(255.0 * o);
    if (qq < 0.0) qq = 0.0;
    double ex = sqrt(qq * S2[0][0]), ey = sqrt(qq * S2[1][1]);
    ext[2 * i] = ex;
    ext[2 * i + 1] = ey;
    valid[i] = 1;
    double u0 = ceil(xy[2 * i] - ex), u1 = floor(xy[2 * i] + ex);
    double v0 = ceil(xy[2 * i + 1] - ey), v1 = floor(xy[2 * i + 1] + ey);
    if (u0 < 0) u0 = 0;
    if (v0 < 0) v0 = 0;
    if (u1 > width - 1) u1 = width - 1;
    if (v1 > height - 1) v1 = height - 1;
    if (u0 > u1 || v0 > v1) continue;
    rect[4 * i + 0] = (int32_t)u0 / tile_w;
    rect[4 * i + 1] = (int32_t)v0 / tile_h;
    rect[4 * i + 2] = (int32_t)u1 / tile_w + 1;
    rect[4 * i + 3] = (int32_t)v1 / tile_h + 1;
    (void)tiles_x;
    (void)tiles_y;
  }
  return 0;
}

/* FP32 image mean of every Gaussian, as a renderer computing in single precision gets
 * it from the FP32 inputs (reading C5: only fused multiply-adds and correctly rounded
 * division, so the value is unique): camera-space t = M p + m as the fma chains
 * t_r = fmaf(M_r0, px, fmaf(M_r1, py, fmaf(M_r2, pz, m_r))), then u = t_x / t_z,
 * v = t_y / t_z, x = fmaf(fx, u, cx), y = fmaf(fy, v, cy).  means: FP32 [3][n];
 * out: FP32 [n][2].  Gaussians behind the camera get whatever the formula gives. */
void or_mean2d_f32(int64_t n, const float* means, const float* viewmat, const float* intr, float* out) {
  for (int64_t i = 0; i < n; ++i) {
    const float px = means[i], py = means[n + i], pz = means[2 * n + i];
    const float tx = fmaf(viewmat[0], px, fmaf(viewmat[1], py, fmaf(viewmat[2], pz, viewmat[3])));
    const float ty = fmaf(viewmat[4], px, fmaf(viewmat[5], py, fmaf(viewmat[6], pz, viewmat[7])));
    const float tz = fmaf(viewmat[8], px, fmaf(viewmat[9], py, fmaf(viewmat[10], pz, viewmat[11])));
    const float u = tx / tz, v = ty / tz;
    out[2 * i] = fmaf(intr[0], u, intr[2]);
    out[2 * i + 1] = fmaf(intr[1], v, intr[3]);
  }
}

/* ------------------------------------------------------------------ */
/* Per-pixel compositing, Eq. (render-gs), with the importance max of  */
/* Eq. (importance-score).                                             */
/* ------------------------------------------------------------------ */

typedef struct {
  float depth;
  int64_t id;
  double alpha;    /* min(0.99, araw) */
  double araw;     /* o * exp(power) */
  double power;
  double araw2;    /* the same at the alternative image mean (= araw without one) */
  double power2;
} or_entry;

static int entry_cmp(const void* a, const void* b) {
  const or_entry* x = (const or_entry*)a;
  const or_entry* y = (const or_entry*)b;
  if (x->depth < y->depth) return -1;
  if (x->depth > y->depth) return 1;
  return (x->id < y->id) ? -1 : (x->id > y->id ? 1 : 0);
}

/* Render the listed pixels (all pixels, row-major, if pix == NULL).
 * mode 0: every valid Gaussian is a candidate for every pixel (brute force).
 * mode 1: candidates come from 16x16-pixel cells listing each Gaussian whose
 *         support bounding box (slightly widened) overlaps the cell; this is a
 *         superset of the alpha >= 1/255 set, so the result is identical.
 * Per pixel: image[3], T_final, last_id (id of the last composited entry, -1 if
 * none), n_contrib, ambiguous: 1 if, before compositing stops, a skip or stop decision
 * lies within a relative amb_rel of its threshold, or 0 < |power| <= 1e-9 -- each
 * decision evaluated at the FP64 image mean xy and, if xy_alt is given, also at xy_alt
 * (the FP32 mean a single-precision renderer uses), where the two evaluations falling on
 * different sides flags the pixel too.  The compositing itself uses xy only.
 * T_amb (may be NULL): the transmittance in front of the first flagged decision (0 for an
 * unflagged pixel); c_amb (may be NULL): the largest colour channel (or background) of
 * the entries from that decision on (0 if unflagged).  Two renderers that agree on every
 * decision before it composite the same front part, and each composites at most
 * T_amb * c_amb behind it, so their images differ by at most that plus rounding.
 * Per Gaussian (in/out, max-accumulated): h, alpha*T of every composited entry that
 * precedes the pixel's first near-threshold decision (an unflagged pixel has none);
 * h_amb, alpha*T of every entry from that decision up to and including the stopping
 * one (entries skipped only by a near-threshold alpha included), which a different
 * rounding of the decision could change.
 * Returns 0, or -1 on allocation failure. */
int or_render(int64_t n, const double* xy, const double* conic, const double* opacity,
              const double* rgb, const float* depth, const int32_t* valid, const double* ext,
              int width, int height, const double* bg, int64_t n_pix, const int32_t* pix, int mode,
              double amb_rel, const double* xy_alt, double* image, double* T_final, int32_t* last_id,
              int32_t* n_contrib, uint8_t* ambiguous, double* T_amb, double* c_amb, double* h, double* h_amb,
              int n_threads) {
  const int CELL = 16;
  const int cells_x = (width + CELL - 1) / CELL, cells_y = (height + CELL - 1) / CELL;
  int64_t* cell_start = NULL;
  int64_t* cell_list = NULL;
  if (mode == 1) {
    cell_start = (int64_t*)calloc((size_t)cells_x * cells_y + 1, sizeof(int64_t));
    if (!cell_start) return -1;
    for (int pass = 0; pass < 2; ++pass) {
      int64_t* fill = NULL;
      if (pass == 1) {
        for (int64_t c = 0; c < (int64_t)cells_x * cells_y; ++c) cell_start[c + 1] += cell_start[c];
        cell_list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cell_start[(int64_t)cells_x * cells_y] + 1));
        fill = (int64_t*)calloc((size_t)cells_x * cells_y, sizeof(int64_t));
        if (!cell_list || !fill) return -1;
      }
      for (int64_t i = 0; i < n; ++i) {
        if (!valid[i]) continue;
        /* widened so that the FP64 alpha test never keeps a pixel outside the box */
        double mx = ext[2 * i] * (1.0 + 1e-6) + 1e-6, my = ext[2 * i + 1] * (1.0 + 1e-6) + 1e-6;
        if (xy_alt) {   /* cover the support around either mean */
          mx += fabs(xy_alt[2 * i] - xy[2 * i]);
          my += fabs(xy_alt[2 * i + 1] - xy[2 * i + 1]);
        }
        double u0 = ceil(xy[2 * i] - mx), u1 = floor(xy[2 * i] + mx);
        double v0 = ceil(xy[2 * i + 1] - my), v1 = floor(xy[2 * i + 1] + my);
        if (u0 < 0) u0 = 0;
        if (v0 < 0) v0 = 0;
        if (u1 > width - 1) u1 = width - 1;
        if (v1 > height - 1) v1 = height - 1;
        if (u0 > u1 || v0 > v1) continue;
        for (int cyy = (int)v0 / CELL; cyy <= (int)v1 / CELL; ++cyy)
          for (int cxx = (int)u0 / CELL; cxx <= (int)u1 / CELL; ++cxx) {
            int64_t c = (int64_t)cyy * cells_x + cxx;
            if (pass == 0) cell_start[c + 1] += 1;
            else cell_list[cell_start[c] + fill[c]++] = i;
          }
      }
      if (pass == 1) free(fill);
    }
  }
  const int64_t total = pix ? n_pix : (int64_t)width * height;
  const double a_lo = OR_ALPHA_MIN * (1.0 - amb_rel);
  int fail = 0;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
  {
    int64_t cap = 1024;
    or_entry* ent = (or_entry*)malloc(sizeof(or_entry) * cap);
    int64_t* hid = (int64_t*)malloc(sizeof(int64_t) * cap);
    double* hval = (double*)malloc(sizeof(double) * cap);
    int64_t* hpos = (int64_t*)malloc(sizeof(int64_t) * cap);
    if (!ent || !hid || !hval || !hpos) fail = 1;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
    for (int64_t k = 0; k < total; ++k) {
      if (fail) continue;
      int u = pix ? pix[2 * k] : (int)(k % width);
      int v = pix ? pix[2 * k + 1] : (int)(k / width);
      int64_t ncand;
      const int64_t* cand = NULL;
      if (mode == 1) {
        int64_t c = (int64_t)(v / CELL) * cells_x + (u / CELL);
        cand = cell_list + cell_start[c];
        ncand = cell_start[c + 1] - cell_start[c];
      } else {
        ncand = n;
      }
      /* candidates that are kept, or that a near-threshold decision could keep */
      int64_t ne = 0;
      for (int64_t t = 0; t < ncand; ++t) {
        int64_t j = cand ? cand[t] : t;
        if (!valid[j]) continue;
        double dx = (double)u - xy[2 * j], dy = (double)v - xy[2 * j + 1];
        double power = -0.5 * (conic[3 * j] * dx * dx + conic[3 * j + 2] * dy * dy) -
                       conic[3 * j + 1] * dx * dy;
        double araw = opacity[j] * exp(power);
        double power2 = power, araw2 = araw;
        if (xy_alt) {
          double dx2 = (double)u - xy_alt[2 * j], dy2 = (double)v - xy_alt[2 * j + 1];
          power2 = -0.5 * (conic[3 * j] * dx2 * dx2 + conic[3 * j + 2] * dy2 * dy2) - conic[3 * j + 1] * dx2 * dy2;
          araw2 = opacity[j] * exp(power2);
        }
        /* an entry neither evaluation could keep changes nothing */
        if ((power > 1e-9 || araw < a_lo) && (power2 > 1e-9 || araw2 < a_lo)) continue;
        if (ne == cap) {
          cap *= 2;
          ent = (or_entry*)realloc(ent, sizeof(or_entry) * cap);
          hid = (int64_t*)realloc(hid, sizeof(int64_t) * cap);
          hval = (double*)realloc(hval, sizeof(double) * cap);
          hpos = (int64_t*)realloc(hpos, sizeof(int64_t) * cap);
          if (!ent || !hid || !hval || !hpos) { fail = 1; break; }
        }
        ent[ne].depth = depth[j];
        ent[ne].id = j;
        ent[ne].araw = araw;
        ent[ne].alpha = araw < OR_ALPHA_MAX ? araw : OR_ALPHA_MAX;
        ent[ne].power = power;
        ent[ne].araw2 = araw2;
        ent[ne].power2 = power2;
        ++ne;
      }
      if (fail) continue;
      qsort(ent, (size_t)ne, sizeof(or_entry), entry_cmp);
      double T = 1.0, C[3] = {0.0, 0.0, 0.0};
      double T2 = 1.0;       /* transmittance from the alternative alphas, up to the first flag */
      double Tat = 0.0;      /* transmittance in front of the first flagged decision */
      int64_t last = -1, cnt = 0, stop = ne;
      int64_t amb_at = -1;   /* sorted position of the first near-threshold decision */
      for (int64_t e = 0; e < ne; ++e) {
        const double p1 = ent[e].power, p2 = ent[e].power2;
        const double r1 = ent[e].araw, r2 = ent[e].araw2;
        if (amb_at < 0) {
          int flag = (p1 != 0.0 && fabs(p1) <= 1e-9) || (p2 != 0.0 && fabs(p2) <= 1e-9) || ((p1 > 0.0) != (p2 > 0.0));
          flag = flag || fabs(r1 - OR_ALPHA_MIN) <= amb_rel * OR_ALPHA_MIN ||
                 fabs(r2 - OR_ALPHA_MIN) <= amb_rel * OR_ALPHA_MIN || ((r1 < OR_ALPHA_MIN) != (r2 < OR_ALPHA_MIN));
          if (flag) { amb_at = e; Tat = T; }
        }
        if (p1 > 0.0) continue;
        double a = ent[e].alpha;
        if (a < OR_ALPHA_MIN) continue;
        double Tn = T * (1.0 - a);
        if (amb_at < 0) {
          const double a2 = r2 < OR_ALPHA_MAX ? r2 : OR_ALPHA_MAX;
          const double Tn2 = T2 * (1.0 - a2);
          if (fabs(Tn - OR_T_MIN) <= amb_rel * OR_T_MIN || fabs(Tn2 - OR_T_MIN) <= amb_rel * OR_T_MIN ||
              ((Tn < OR_T_MIN) != (Tn2 < OR_T_MIN))) {
            amb_at = e;
            Tat = T;
          }
          T2 = Tn2;
        }
        if (Tn < OR_T_MIN) { stop = e; break; }
        const double* c = rgb + 3 * ent[e].id;
        C[0] += c[0] * a * T;
        C[1] += c[1] * a * T;
        C[2] += c[2] * a * T;
        hid[cnt] = ent[e].id;
        hval[cnt] = a * T;
        hpos[cnt] = e;
        T = Tn;
        last = ent[e].id;
        ++cnt;
      }
      if (T_amb) T_amb[k] = amb_at >= 0 ? Tat : 0.0;
      if (c_amb) {
        double cm = 0.0;
        if (amb_at >= 0) {
          for (int ch = 0; ch < 3; ++ch) {
            const double b = bg ? fabs(bg[ch]) : 0.0;
            if (b > cm) cm = b;
          }
          for (int64_t e = amb_at; e < ne; ++e)
            for (int ch = 0; ch < 3; ++ch)
              if (rgb[3 * ent[e].id + ch] > cm) cm = rgb[3 * ent[e].id + ch];
        }
        c_amb[k] = cm;
      }
      const int amb = amb_at >= 0;
      for (int ch = 0; ch < 3; ++ch) image[3 * k + ch] = C[ch] + T * (bg ? bg[ch] : 0.0);
      T_final[k] = T;
      last_id[k] = (int32_t)last;
      n_contrib[k] = (int32_t)cnt;
      ambiguous[k] = (uint8_t)amb;
#ifdef _OPENMP
#pragma omp critical(or_importance)
#endif
      {
        /* entries composited before the first near-threshold decision are unaffected by
           how that decision falls; the rest go to h_amb */
        for (int64_t e = 0; e < cnt; ++e)
          if ((!amb || hpos[e] < amb_at) && hval[e] > h[hid[e]]) h[hid[e]] = hval[e];
        if (amb && h_amb) {
          double Tp = 1.0;
          for (int64_t e = 0; e < ne && e <= stop; ++e) {
            double val = ent[e].alpha * Tp;
            if (e >= amb_at && val > h_amb[ent[e].id]) h_amb[ent[e].id] = val;
            if (ent[e].power <= 0.0 && ent[e].alpha >= OR_ALPHA_MIN) Tp *= (1.0 - ent[e].alpha);
          }
        }
      }
    }
    free(ent);
    free(hid);
    free(hval);
    free(hpos);
  }
  free(cell_start);
  free(cell_list);
  return fail ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Integer stages: duplicated (tile | depth) keys, stable sort, ranges. */
/* ------------------------------------------------------------------ */

typedef struct {
  uint64_t key;
  uint32_t val;
  int64_t seq;
} or_kv;

static int kv_cmp(const void* a, const void* b) {
  const or_kv* x = (const or_kv*)a;
  const or_kv* y = (const or_kv*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->seq < y->seq ? -1 : (x->seq > y->seq ? 1 : 0);
}

/* For items 0..m-1 in increasing order, and for each tile of the item's rect in
 * row-major order, emit key = (tile_base[view] + ty*tiles_x[view] + tx) << 32 |
 * bits(depth) and val = item; then sort by key keeping emission order among equal
 * keys.  Returns the number of instances K (keys/vals are written only if K <= cap). */
int64_t or_bin_sort(int64_t m, const float* depth, const uint16_t* rect, const int32_t* item_view,
                    const int32_t* view_tiles_x, const int32_t* view_tile_base, int64_t cap,
                    uint64_t* keys, uint32_t* vals) {
  int64_t K = 0;
  for (int64_t i = 0; i < m; ++i) {
    int64_t w = (int64_t)rect[4 * i + 2] - rect[4 * i + 0];
    int64_t h = (int64_t)rect[4 * i + 3] - rect[4 * i + 1];
    if (w > 0 && h > 0) K += w * h;
  }
  if (K > cap) return K;
  or_kv* kv = (or_kv*)malloc(sizeof(or_kv) * (size_t)(K > 0 ? K : 1));
  if (!kv) return -1;
  int64_t k = 0;
  for (int64_t i = 0; i < m; ++i) {
    uint32_t dbits;
    memcpy(&dbits, &depth[i], sizeof(dbits));
    int v = item_view[i];
    for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty)
      for (int tx = rect[4 * i + 0]; tx < rect[4 * i + 2]; ++tx) {
        uint64_t tile = (uint64_t)view_tile_base[v] + (uint64_t)ty * view_tiles_x[v] + tx;
        kv[k].key = (tile << 32) | dbits;
        kv[k].val = (uint32_t)i;
        kv[k].seq = k;
        ++k;
      }
  }
  qsort(kv, (size_t)K, sizeof(or_kv), kv_cmp);
  for (int64_t e = 0; e < K; ++e) {
    keys[e] = kv[e].key;
    vals[e] = kv[e].val;
  }
  free(kv);
  return K;
}

/* ranges[2t], ranges[2t+1] = first and one-past-last position of tile t in the
 * sorted keys: the number of instances on tiles < t and on tiles <= t.  A tile with
 * no instance gets the empty range [s, s) at the place its list would start (reading
 * C5: that position is unique, so empty tiles are compared bit for bit too). */
void or_tile_ranges(int64_t K, const uint64_t* keys, int64_t n_tiles, uint32_t* ranges) {
  int64_t e = 0;
  for (int64_t t = 0; t < n_tiles; ++t) {
    ranges[2 * t] = (uint32_t)e;
    while (e < K && (int64_t)(keys[e] >> 32) == t) ++e;
    ranges[2 * t + 1] = (uint32_t)e;
  }
}

/* ------------------------------------------------------------------ */
/* Pruning / visibility masks (Sec. 3.3, Eq. importance-score-vis)     */
/* and the nearest cluster centre (Sec. 3.4).                          */
/* ------------------------------------------------------------------ */

/* mode 0: mask = h < t (points the pruning step removes);
 * mode 1: mask = h > t (points visible for a cluster).
 * idx lists the masked indices in ascending order; returns their count. */
int64_t or_filter(int64_t n, const float* h, float t, int mode, uint8_t* mask, uint32_t* idx) {
  int64_t cnt = 0;
  for (int64_t i = 0; i < n; ++i) {
    /* mode 0: the pruning mask 1(h < t) (Sec. 3.3); 1: the visibility indicator 1(h > t)
     * (Eq. importance-score-vis); 2: the points pruning keeps, 1(h >= t) = 1 - mode 0 */
    int on = mode == 0 ? (h[i] < t) : mode == 1 ? (h[i] > t) : (h[i] >= t);
    mask[i] = (uint8_t)on;
    if (on) idx[cnt++] = (uint32_t)i;
  }
  return cnt;
}

/* For each camera centre, the index of the nearest of k centres; the squared
 * distance is ((x0-c0)^2 + (x1-c1)^2) + (x2-c2)^2 in FP32, lowest index wins ties. */
void or_nearest(int32_t k, const float* centres, int32_t n_cams, const float* cams, int32_t* out) {
  for (int32_t c = 0; c < n_cams; ++c) {
    int32_t best = -1;
    float bd = 0.0f;
    for (int32_t j = 0; j < k; ++j) {
      float d0 = cams[3 * c] - centres[3 * j];
      float d1 = cams[3 * c + 1] - centres[3 * j + 1];
      float d2 = cams[3 * c + 2] - centres[3 * j + 2];
      float d = d0 * d0;
      d = d + d1 * d1;
      d = d + d2 * d2;
      if (best < 0 || d < bd) {
        best = j;
        bd = d;
      }
    }
    out[c] = best;
  }
}
