/*
 * disk_oracle.c -- plain, slow FP64 CPU oracle for DISK (Differentiable Sparse
 * Kernel Complex, arXiv 2512.04556).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header or constant table with the CUDA
 * library; the two meet only through the seeded input arrays.
 *
 * Every routine is the paper's definition written out in FP64 with no blocking,
 * fusion or reordering beyond what the definition states.  Where the paper is
 * silent, the reading taken is stated at the routine.
 *
 * Conventions (shared by name, not by code, with the library):
 *   image      double [H][W][C] row-major, pixel (v,u) = (row, column)
 *   map        double [dims][H][W]  raw kernel-space parameter p(x)
 *   offset     o = (dx, dy): dx along columns (u), dy along rows (v), pixels
 *   theta      double [B][L][T][3] = (dx, dy, w) per node, layer, tap
 *   2-D basis  node (a, b) has index a * n_nodes[1] + b; axis 0 is map 0
 *   boundary   0 = clamp-to-edge (image filtering), 1 = zero outside (impulse
 *              synthesis on a canvas)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the state advances by the golden-ratio increment
 * and each output is the state passed through the variant-13 finaliser. */
uint64_t orc_splitmix64(uint64_t *state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Uniform double in [0,1) from the top 53 bits of one SplitMix64 output. */
static double orc_uniform(uint64_t *state) {
  return (double)(orc_splitmix64(state) >> 11) * (1.0 / 9007199254740992.0);
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ------------------------------------------------------------------------- */
/* Filter-space interpolation weights, Sec. 4.3 Eq. 8-9.                      */
/* ------------------------------------------------------------------------- */

/* Locate p among increasing nodes[0..n-1]: lower node k and blend t such that
 * the two non-zero weights are alpha_k = 1-t, alpha_{k+1} = t (linear
 * interpolation between adjacent nodes, a convex combination as Eq. 9
 * requires).  p is clamped to [nodes[0], nodes[n-1]]; at the top node k = n-2,
 * t = 1.  A non-finite p is treated as nodes[0]. */
void orc_locate(double p, const double *nodes, int n, int *k, double *t) {
  if (n <= 1) { *k = 0; *t = 0.0; return; }
  if (!(p > nodes[0])) { *k = 0; *t = 0.0; return; }      /* also catches NaN */
  if (p >= nodes[n - 1]) { *k = n - 2; *t = 1.0; return; }
  int j = 0;
  while (j < n - 2 && p > nodes[j + 1]) j++;
  *k = j;
  *t = (p - nodes[j]) / (nodes[j + 1] - nodes[j]);
}

/* Full weight vector alpha[B] for the parameter values pv[dims] (Eq. 9).
 * 1-D: two neighbours.  2-D: tensor product of the per-axis weights. */
void orc_alpha(const double *pv, int dims, const int *n_nodes,
               const double *node_vals, double *alpha) {
  if (dims == 1) {
    int n = n_nodes[0], k; double t;
    for (int i = 0; i < n; i++) alpha[i] = 0.0;
    orc_locate(pv[0], node_vals, n, &k, &t);
    if (n == 1) { alpha[0] = 1.0; return; }
    alpha[k] += 1.0 - t;
    alpha[k + 1] += t;
  } else {
    int n0 = n_nodes[0], n1 = n_nodes[1];
    double a0[4096], a1[4096];
    int k; double t;
    for (int i = 0; i < n0; i++) a0[i] = 0.0;
    for (int i = 0; i < n1; i++) a1[i] = 0.0;
    orc_locate(pv[0], node_vals, n0, &k, &t);
    if (n0 == 1) a0[0] = 1.0; else { a0[k] += 1.0 - t; a0[k + 1] += t; }
    orc_locate(pv[1], node_vals + n0, n1, &k, &t);
    if (n1 == 1) a1[0] = 1.0; else { a1[k] += 1.0 - t; a1[k + 1] += t; }
    for (int a = 0; a < n0; a++)
      for (int b = 0; b < n1; b++) alpha[a * n1 + b] = a0[a] * a1[b];
  }
}

/* Eq. 9 applied to offsets and weights alike: taps[L][T][3] = sum_k alpha_k
 * theta_k, summed over every node in index order. */
void orc_blend(const double *alpha, int B, int L, int T, const double *theta,
               double *taps) {
  int n = L * T * 3;
  for (int j = 0; j < n; j++) taps[j] = 0.0;
  for (int k = 0; k < B; k++) {
    if (alpha[k] == 0.0) continue;
    for (int j = 0; j < n; j++) taps[j] += alpha[k] * theta[(long)k * n + j];
  }
}

/* ------------------------------------------------------------------------- */
/* One sparse tap (Eq. 2) with bilinear sampling at a fractional offset.      */
/* ------------------------------------------------------------------------- */

static double fetch(const double *img, int H, int W, int C, int y, int x, int c,
                    int boundary) {
  if (boundary == 0) {
    y = clampi(y, 0, H - 1);
    x = clampi(x, 0, W - 1);
  } else if (y < 0 || y >= H || x < 0 || x >= W) {
    return 0.0;
  }
  return img[((long)y * W + x) * C + c];
}

/* Bilinear sample of channel c at (v + dy, u + dx).  Texel centres sit at
 * integer coordinates; the integer and fractional parts come from the offset
 * alone (ix = u + floor(dx), fx = dx - floor(dx)).  Optionally returns the
 * partial derivatives with respect to dx and dy (one-sided at integers). */
double orc_bilinear(const double *img, int H, int W, int C, int c, int v, int u,
                    double dx, double dy, int boundary, double *d_dx,
                    double *d_dy) {
  double flx = floor(dx), fly = floor(dy);
  double fx = dx - flx, fy = dy - fly;
  int ix = u + (int)flx, iy = v + (int)fly;
  double a = fetch(img, H, W, C, iy, ix, c, boundary);
  double b = fetch(img, H, W, C, iy, ix + 1, c, boundary);
  double cc = fetch(img, H, W, C, iy + 1, ix, c, boundary);
  double d = fetch(img, H, W, C, iy + 1, ix + 1, c, boundary);
  if (d_dx) *d_dx = (1.0 - fy) * (b - a) + fy * (d - cc);
  if (d_dy) *d_dy = (1.0 - fx) * (cc - a) + fx * (d - b);
  return (1.0 - fx) * (1.0 - fy) * a + fx * (1.0 - fy) * b +
         (1.0 - fx) * fy * cc + fx * fy * d;
}

/* One layer of the cascade, Eq. 3: out[x] = sum_i w_i * sample(in, x + o_i).
 * taps points at T*3 values per pixel when tap_stride is T*3 (spatially
 * varying) or at one shared set when tap_stride is 0 (shift invariant). */
void orc_layer(const double *in, double *out, int H, int W, int C, int T,
               const double *taps, long tap_stride, int boundary) {
#pragma omp parallel for schedule(static)
  for (int v = 0; v < H; v++) {
    for (int u = 0; u < W; u++) {
      const double *tp = taps + ((long)v * W + u) * tap_stride;
      for (int c = 0; c < C; c++) {
        double acc = 0.0;
        for (int i = 0; i < T; i++)
          acc += tp[3 * i + 2] *
                 orc_bilinear(in, H, W, C, c, v, u, tp[3 * i], tp[3 * i + 1],
                              boundary, NULL, NULL);
        out[((long)v * W + u) * C + c] = acc;
      }
    }
  }
}

/* Per-pixel blended taps for layer l of a basis (Eq. 9 evaluated at the
 * pixel's own map values).  taps_out[H*W][T][3]. */
static void sv_layer_taps(const double *maps, int H, int W, int dims,
                          const int *n_nodes, const double *node_vals, int L,
                          int T, const double *theta, int l, double *taps_out) {
  int B = dims == 1 ? n_nodes[0] : n_nodes[0] * n_nodes[1];
  long HW = (long)H * W;
#pragma omp parallel
  {
    double *alpha = (double *)malloc(sizeof(double) * B);
    double *all = (double *)malloc(sizeof(double) * L * T * 3);
#pragma omp for schedule(static)
    for (long px = 0; px < HW; px++) {
      double pv[2];
      pv[0] = maps[px];
      pv[1] = dims == 2 ? maps[HW + px] : 0.0;
      orc_alpha(pv, dims, n_nodes, node_vals, alpha);
      orc_blend(alpha, B, L, T, theta, all);
      memcpy(taps_out + px * T * 3, all + (long)l * T * 3, sizeof(double) * T * 3);
    }
    free(alpha);
    free(all);
  }
}

/* Spatially varying filter, Eq. 3 with the per-pixel complex of Eq. 9: every
 * layer at output pixel x uses the taps interpolated at x's own parameter
 * values; clamp-to-edge at the image border. */
int orc_sv_filter(const double *img, int H, int W, int C, const double *maps,
                  int dims, const int *n_nodes, const double *node_vals, int L,
                  int T, const double *theta, double *out) {
  if (H <= 0 || W <= 0 || C <= 0 || L <= 0 || T <= 0 || (dims != 1 && dims != 2))
    return ORC_EINVAL;
  long n = (long)H * W * C;
  double *a = (double *)malloc(sizeof(double) * n);
  double *b = (double *)malloc(sizeof(double) * n);
  double *taps = (double *)malloc(sizeof(double) * (long)H * W * T * 3);
  if (!a || !b || !taps) { free(a); free(b); free(taps); return ORC_ENOMEM; }
  memcpy(a, img, sizeof(double) * n);
  for (int l = 0; l < L; l++) {
    sv_layer_taps(maps, H, W, dims, n_nodes, node_vals, L, T, theta, l, taps);
    orc_layer(a, b, H, W, C, T, taps, (long)T * 3, 0);
    double *s = a; a = b; b = s;
  }
  memcpy(out, a, sizeof(double) * n);
  free(a); free(b); free(taps);
  return ORC_OK;
}

/* Spatially varying filter with a per-pixel rotation of the complex: as
 * orc_sv_filter, but after the Eq. 9 blend every tap offset of pixel x is
 * rotated by angle[x] (radians; x right, y down):
 *   (dx, dy) -> (dx cos a - dy sin a, dx sin a + dy cos a).
 * Rotating every offset of every layer rotates the impulse response (Eq. 10)
 * of a shift-invariant complex by the same angle, which is how the 2-D
 * effects of Sec. 5.3 (rotational and radial blur: strength and local blur
 * angle) reduce to a basis over strength alone.  A non-finite angle acts as
 * zero. */
int orc_sv_filter_rot(const double *img, int H, int W, int C, const double *maps,
                      const double *angle, int dims, const int *n_nodes,
                      const double *node_vals, int L, int T, const double *theta,
                      double *out) {
  if (H <= 0 || W <= 0 || C <= 0 || L <= 0 || T <= 0 || (dims != 1 && dims != 2))
    return ORC_EINVAL;
  long n = (long)H * W * C, HW = (long)H * W;
  double *a = (double *)malloc(sizeof(double) * n);
  double *b = (double *)malloc(sizeof(double) * n);
  double *taps = (double *)malloc(sizeof(double) * HW * T * 3);
  if (!a || !b || !taps) { free(a); free(b); free(taps); return ORC_ENOMEM; }
  memcpy(a, img, sizeof(double) * n);
  for (int l = 0; l < L; l++) {
    sv_layer_taps(maps, H, W, dims, n_nodes, node_vals, L, T, theta, l, taps);
    for (long px = 0; px < HW; px++) {
      double phi = isfinite(angle[px]) ? angle[px] : 0.0;
      double cs = cos(phi), sn = sin(phi);
      for (int i = 0; i < T; i++) {
        double *t = taps + (px * T + i) * 3;
        double dx = t[0], dy = t[1];
        t[0] = dx * cs - dy * sn;
        t[1] = dx * sn + dy * cs;
      }
    }
    orc_layer(a, b, H, W, C, T, taps, (long)T * 3, 0);
    double *s = a; a = b; b = s;
  }
  memcpy(out, a, sizeof(double) * n);
  free(a); free(b); free(taps);
  return ORC_OK;
}

/* Adjoint of orc_sv_filter with respect to the image: g_in = F^T g_out.
 * Written as the literal transpose of each layer -- every (pixel, tap,
 * corner) product of the forward pass scatters its weight back onto the
 * (clamped) corner pixel it read. */
int orc_sv_filter_adjoint(const double *g_out, int H, int W, int C,
                          const double *maps, int dims, const int *n_nodes,
                          const double *node_vals, int L, int T,
                          const double *theta, double *g_in) {
  if (H <= 0 || W <= 0 || C <= 0 || L <= 0 || T <= 0 || (dims != 1 && dims != 2))
    return ORC_EINVAL;
  long n = (long)H * W * C;
  double *g = (double *)malloc(sizeof(double) * n);
  double *gp = (double *)malloc(sizeof(double) * n);
  double *taps = (double *)malloc(sizeof(double) * (long)H * W * T * 3);
  if (!g || !gp || !taps) { free(g); free(gp); free(taps); return ORC_ENOMEM; }
  memcpy(g, g_out, sizeof(double) * n);
  for (int l = L - 1; l >= 0; l--) {
    sv_layer_taps(maps, H, W, dims, n_nodes, node_vals, L, T, theta, l, taps);
    memset(gp, 0, sizeof(double) * n);
    for (int v = 0; v < H; v++)
      for (int u = 0; u < W; u++) {
        const double *tp = taps + ((long)v * W + u) * T * 3;
        for (int i = 0; i < T; i++) {
          double dx = tp[3 * i], dy = tp[3 * i + 1], w = tp[3 * i + 2];
          double flx = floor(dx), fly = floor(dy);
          double fx = dx - flx, fy = dy - fly;
          int ix = u + (int)flx, iy = v + (int)fly;
          double beta[4] = {(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy};
          int cy[4] = {iy, iy, iy + 1, iy + 1}, cx[4] = {ix, ix + 1, ix, ix + 1};
          for (int q = 0; q < 4; q++) {
            int yy = clampi(cy[q], 0, H - 1), xx = clampi(cx[q], 0, W - 1);
            for (int c = 0; c < C; c++)
              gp[((long)yy * W + xx) * C + c] +=
                  w * beta[q] * g[((long)v * W + u) * C + c];
          }
        }
      }
    double *s = g; g = gp; gp = s;
  }
  memcpy(g_in, g, sizeof(double) * n);
  free(g); free(gp); free(taps);
  return ORC_OK;
}


/* Gradient of L = <g_out, F(img)> with respect to the basis theta, through
 * the spatially varying cascade: each layer's per-pixel tap (Eq. 9 blend at
 * the pixel) receives dL/dw = sum_c G_l[x,c] s_c and dL/d(dx,dy) =
 * w sum_c G_l[x,c] ds_c/d(dx,dy) with s the bilinear sample of the layer
 * input, and passes it to node k with weight alpha_k(x) (Eq. 9 is linear in
 * theta).  G_{l-1} is the transpose of layer l applied to G_l, as in
 * orc_sv_filter_adjoint.  grad_theta [B][L][T][3] is overwritten. */
int orc_sv_filter_grad_theta(const double *img, const double *g_out, int H, int W, int C,
                             const double *maps, int dims, const int *n_nodes,
                             const double *node_vals, int L, int T, const double *theta,
                             double *grad_theta) {
  if (H <= 0 || W <= 0 || C <= 0 || L <= 0 || T <= 0 || (dims != 1 && dims != 2))
    return ORC_EINVAL;
  int B = dims == 1 ? n_nodes[0] : n_nodes[0] * n_nodes[1];
  long HW = (long)H * W, n = HW * C;
  double *acts = (double *)malloc(sizeof(double) * n * L);
  double *g = (double *)malloc(sizeof(double) * n);
  double *gp = (double *)malloc(sizeof(double) * n);
  double *taps = (double *)malloc(sizeof(double) * HW * T * 3);
  double *alpha = (double *)malloc(sizeof(double) * HW * B);
  if (!acts || !g || !gp || !taps || !alpha) {
    free(acts); free(g); free(gp); free(taps); free(alpha);
    return ORC_ENOMEM;
  }
  for (long px = 0; px < HW; px++) {
    double pv[2] = {maps[px], dims == 2 ? maps[HW + px] : 0.0};
    orc_alpha(pv, dims, n_nodes, node_vals, alpha + px * B);
  }
  /* forward, keeping every layer's input */
  memcpy(acts, img, sizeof(double) * n);
  for (int l = 0; l + 1 < L; l++) {
    sv_layer_taps(maps, H, W, dims, n_nodes, node_vals, L, T, theta, l, taps);
    orc_layer(acts + (long)l * n, acts + (long)(l + 1) * n, H, W, C, T, taps, (long)T * 3, 0);
  }
  memset(grad_theta, 0, sizeof(double) * (size_t)B * L * T * 3);
  memcpy(g, g_out, sizeof(double) * n);
  for (int l = L - 1; l >= 0; l--) {
    const double *in = acts + (long)l * n;
    sv_layer_taps(maps, H, W, dims, n_nodes, node_vals, L, T, theta, l, taps);
    memset(gp, 0, sizeof(double) * n);
    for (int v = 0; v < H; v++)
      for (int u = 0; u < W; u++) {
        long px = (long)v * W + u;
        const double *tp = taps + px * T * 3;
        for (int i = 0; i < T; i++) {
          double dx = tp[3 * i], dy = tp[3 * i + 1], w = tp[3 * i + 2];
          double gw = 0, gdx = 0, gdy = 0;
          for (int c = 0; c < C; c++) {
            double sdx, sdy;
            double sv = orc_bilinear(in, H, W, C, c, v, u, dx, dy, 0, &sdx, &sdy);
            double gc = g[px * C + c];
            gw += gc * sv; gdx += gc * w * sdx; gdy += gc * w * sdy;
          }
          for (int k = 0; k < B; k++) {
            double a = alpha[px * B + k];
            if (a == 0.0) continue;
            double *gt = grad_theta + (((size_t)k * L + l) * T + i) * 3;
            gt[0] += a * gdx; gt[1] += a * gdy; gt[2] += a * gw;
          }
          double flx = floor(dx), fly = floor(dy);
          double fx = dx - flx, fy = dy - fly;
          int ix = u + (int)flx, iy = v + (int)fly;
          double beta[4] = {(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy};
          int cy[4] = {iy, iy, iy + 1, iy + 1}, cx[4] = {ix, ix + 1, ix, ix + 1};
          for (int q = 0; q < 4; q++) {
            int yy = clampi(cy[q], 0, H - 1), xx = clampi(cx[q], 0, W - 1);
            for (int c = 0; c < C; c++)
              gp[((long)yy * W + xx) * C + c] += w * beta[q] * g[px * C + c];
          }
        }
      }
    double *t = g; g = gp; gp = t;
  }
  free(acts); free(g); free(gp); free(taps); free(alpha);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Impulse-response synthesis, Sec. 4.4 Eq. 10 (composite kernel of Eq. 4).  */
/* ------------------------------------------------------------------------- */

/* Half-width, in pixels, that holds the whole impulse response of a shift-
 * invariant complex: each layer widens the support by ceil(max |o|) + 1
 * (the +1 is the bilinear footprint). */
int orc_support_radius(const double *theta, int L, int T) {
  int R = 0;
  for (int l = 0; l < L; l++) {
    double m = 0.0;
    for (int i = 0; i < T; i++) {
      double ax = fabs(theta[(l * T + i) * 3]), ay = fabs(theta[(l * T + i) * 3 + 1]);
      if (ax > m) m = ax;
      if (ay > m) m = ay;
    }
    R += (int)ceil(m) + 1;
  }
  return R;
}

/* Impulse response on a zero-padded canvas of half-width R (side 2R+1): a
 * single 1 at the centre c, then the L shift-invariant layers of theta
 * [L][T][3] with zero outside the canvas.  With R >= orc_support_radius the
 * canvas truncates nothing.  acts, if non-NULL, receives all L+1 planes. */
int orc_synth_canvas(const double *theta, int L, int T, int R, double *out,
                     double *acts) {
  if (L <= 0 || T <= 0 || R < 0) return ORC_EINVAL;
  int N = 2 * R + 1;
  long NN = (long)N * N;
  double *a = (double *)calloc(NN, sizeof(double));
  double *b = (double *)calloc(NN, sizeof(double));
  if (!a || !b) { free(a); free(b); return ORC_ENOMEM; }
  a[(long)R * N + R] = 1.0;
  if (acts) memcpy(acts, a, sizeof(double) * NN);
  for (int l = 0; l < L; l++) {
    orc_layer(a, b, N, N, 1, T, theta + (long)l * T * 3, 0, 1);
    double *s = a; a = b; b = s;
    if (acts) memcpy(acts + (l + 1) * NN, a, sizeof(double) * NN);
  }
  memcpy(out, a, sizeof(double) * NN);
  free(a); free(b);
  return ORC_OK;
}

/* K_syn cropped to K x K about the centre (K odd). */
int orc_synth(const double *theta, int L, int T, int K, double *out) {
  if (K <= 0 || (K & 1) == 0) return ORC_EINVAL;
  int h = (K - 1) / 2, R = orc_support_radius(theta, L, T);
  if (R < h) R = h;
  int N = 2 * R + 1;
  double *canvas = (double *)malloc(sizeof(double) * (long)N * N);
  if (!canvas) return ORC_ENOMEM;
  int rc = orc_synth_canvas(theta, L, T, R, canvas, NULL);
  if (rc == ORC_OK)
    for (int y = 0; y < K; y++)
      for (int x = 0; x < K; x++)
        out[y * K + x] = canvas[(long)(R - h + y) * N + (R - h + x)];
  free(canvas);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Fit objective (Eq. 4 with the impulse supervision of Eq. 10-11) and its    */
/* gradient with respect to every offset and weight (Eq. 5).                 */
/* ------------------------------------------------------------------------- */

/* loss_kind 0 = MSE: sum over the plane of (K_syn - K_tgt)^2 / K^2, target
 * zero-padded.  loss_kind 1 = Charbonnier (Eq. 11): sum of
 * (sqrt(d^2 + eps^2) - eps) / K^2, which is zero where d = 0 so it too is
 * independent of the canvas.  grad[L][T][3] in pixel units if non-NULL. */
double orc_fit_loss(const double *theta, int L, int T, const double *target,
                    int K, int loss_kind, double eps, double *grad) {
  int h = (K - 1) / 2, R = orc_support_radius(theta, L, T);
  if (R < h) R = h;
  int N = 2 * R + 1;
  long NN = (long)N * N;
  double *acts = (double *)malloc(sizeof(double) * NN * (L + 1));
  double *G = (double *)calloc(NN, sizeof(double));
  double *Gp = (double *)calloc(NN, sizeof(double));
  double *tmp = (double *)malloc(sizeof(double) * NN);
  if (!acts || !G || !Gp || !tmp) {
    free(acts); free(G); free(Gp); free(tmp);
    return NAN;
  }
  orc_synth_canvas(theta, L, T, R, tmp, acts);
  const double *Ks = acts + (long)L * NN;
  double inv = 1.0 / ((double)K * K), loss = 0.0;
  for (int y = 0; y < N; y++)
    for (int x = 0; x < N; x++) {
      int ty = y - (R - h), tx = x - (R - h);
      double tv = (ty >= 0 && ty < K && tx >= 0 && tx < K) ? target[ty * K + tx] : 0.0;
      double d = Ks[(long)y * N + x] - tv;
      if (loss_kind == 0) {
        loss += d * d * inv;
        G[(long)y * N + x] = 2.0 * d * inv;
      } else {
        double s = sqrt(d * d + eps * eps);
        loss += (s - eps) * inv;
        G[(long)y * N + x] = d / s * inv;
      }
    }
  if (grad) {
    for (int j = 0; j < L * T * 3; j++) grad[j] = 0.0;
    for (int l = L - 1; l >= 0; l--) {
      const double *prev = acts + (long)l * NN;
      const double *tp = theta + (long)l * T * 3;
      double *gl = grad + (long)l * T * 3;
      memset(Gp, 0, sizeof(double) * NN);
      for (int v = 0; v < N; v++)
        for (int u = 0; u < N; u++) {
          double g = G[(long)v * N + u];
          if (g == 0.0) continue;
          for (int i = 0; i < T; i++) {
            double dx = tp[3 * i], dy = tp[3 * i + 1], w = tp[3 * i + 2];
            double sdx, sdy;
            double s = orc_bilinear(prev, N, N, 1, 0, v, u, dx, dy, 1, &sdx, &sdy);
            gl[3 * i + 2] += g * s;
            gl[3 * i + 0] += g * w * sdx;
            gl[3 * i + 1] += g * w * sdy;
            double flx = floor(dx), fly = floor(dy);
            double fx = dx - flx, fy = dy - fly;
            int ix = u + (int)flx, iy = v + (int)fly;
            double beta[4] = {(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy};
            int cy[4] = {iy, iy, iy + 1, iy + 1}, cx[4] = {ix, ix + 1, ix, ix + 1};
            for (int q = 0; q < 4; q++)
              if (cy[q] >= 0 && cy[q] < N && cx[q] >= 0 && cx[q] < N)
                Gp[(long)cy[q] * N + cx[q]] += g * w * beta[q];
          }
        }
      double *s = G; G = Gp; Gp = s;
    }
  }
  free(acts); free(G); free(Gp); free(tmp);
  return loss;
}

/* ------------------------------------------------------------------------- */
/* Initialisation, Sec. 4.1 Eq. 6 (radial) and Sec. 4.2 Eq. 7 (sparse        */
/* sampling).  theta in pixel units.                                          */
/* ------------------------------------------------------------------------- */

/* Per-axis standard deviation of the target about its centroid. */
static double target_sigma(const double *tgt, int K) {
  double s = 0, mx = 0, my = 0;
  for (int y = 0; y < K; y++)
    for (int x = 0; x < K; x++) { double t = tgt[y * K + x]; s += t; mx += t * x; my += t * y; }
  if (!(s > 0)) return 1.0;
  mx /= s; my /= s;
  double var = 0;
  for (int y = 0; y < K; y++)
    for (int x = 0; x < K; x++) {
      double t = tgt[y * K + x];
      var += t * ((x - mx) * (x - mx) + (y - my) * (y - my));
    }
  return sqrt(var / (2.0 * s));
}

/* Rings of Eq. 6 for layers l0..L-1 (0-based), radius (l - l0 + 1) * dr,
 * angle 2 pi i / T for i = 1..T, weight 1/T. */
static void rings(double *theta, int L, int T, int l0, double dr) {
  for (int l = l0; l < L; l++) {
    double r = (l - l0 + 1) * dr;
    for (int i = 0; i < T; i++) {
      double ang = 2.0 * M_PI * (double)(i + 1) / (double)T;
      theta[(l * T + i) * 3 + 0] = r * cos(ang);
      theta[(l * T + i) * 3 + 1] = r * sin(ang);
      theta[(l * T + i) * 3 + 2] = 1.0 / T;
    }
  }
}

/* Increasing-radial initialisation, Eq. 6.  The appendix that derives the
 * step is not available; the step is chosen so that the composite's second
 * moment matches the target's: a ring of radius r has per-axis variance
 * r^2/2 and layer moments add under convolution, so
 * sum_l (l dr)^2 / 2 = sigma_t^2, i.e. dr = sigma_t sqrt(12 / (L(L+1)(2L+1))). */
void orc_init_ir(const double *tgt, int K, int L, int T, double *theta) {
  double sig = target_sigma(tgt, K);
  double dr = sig * sqrt(12.0 / ((double)L * (L + 1) * (2 * L + 1)));
  rings(theta, L, T, 0, dr);
}

/* Sparse-sampling initialisation, Sec. 4.2.  S = number of non-zero target
 * pixels, r = sqrt(S / (T pi)) (Eq. 7, N_s = layer 1's tap count).  Dart
 * throwing over the non-zero pixels: candidate index = SplitMix64 output mod
 * S, accepted when its squared distance to every accepted sample is >= r^2;
 * after 30*T consecutive rejections r^2 <- 0.81 r^2 (r <- 0.9 r), and once
 * r^2 < 0.25 every candidate is accepted.  Layer 1 taps sit at the negated
 * sample positions (gather convention: the response lands on the samples);
 * layers 2..L are Eq. 6 rings whose second moment equals that of a disk of
 * radius r (the area each sample stands for): dr = r / sqrt(2 sum_{j<L} j^2).
 * Returns the number of candidates drawn. */
long orc_init_ss(const double *tgt, int K, int L, int T, uint64_t seed,
                 double *theta) {
  int h = (K - 1) / 2;
  long S = 0;
  for (long j = 0; j < (long)K * K; j++) if (tgt[j] > 0) S++;
  if (S == 0) { orc_init_ir(tgt, K, L, T, theta); return 0; }
  long *idx = (long *)malloc(sizeof(long) * S);
  long n = 0;
  for (long j = 0; j < (long)K * K; j++) if (tgt[j] > 0) idx[n++] = j;
  double r2 = (double)S / ((double)T * M_PI);
  double r0 = sqrt(r2);
  double *ax = (double *)malloc(sizeof(double) * T), *ay = (double *)malloc(sizeof(double) * T);
  int acc = 0, fails = 0;
  long drawn = 0;
  uint64_t st = seed;
  while (acc < T) {
    uint64_t z = orc_splitmix64(&st);
    drawn++;
    long p = idx[z % (uint64_t)S];
    double qx = (double)(p % K - h), qy = (double)(p / K - h);
    int ok = 1;
    for (int a = 0; a < acc && ok; a++) {
      double ddx = qx - ax[a], ddy = qy - ay[a];
      if (ddx * ddx + ddy * ddy < r2) ok = 0;
    }
    if (ok) { ax[acc] = qx; ay[acc] = qy; acc++; fails = 0; }
    else if (++fails >= 30 * T) { r2 *= 0.81; fails = 0; if (r2 < 0.25) r2 = 0.0; }
  }
  for (int i = 0; i < T; i++) {
    theta[i * 3 + 0] = -ax[i];
    theta[i * 3 + 1] = -ay[i];
    theta[i * 3 + 2] = 1.0 / T;
  }
  if (L > 1) {
    double sj = 0;
    for (int j = 1; j < L; j++) sj += (double)j * j;
    rings(theta, L, T, 1, r0 / sqrt(2.0 * sj));
  }
  free(idx); free(ax); free(ay);
  return drawn;
}

/* Random initialisation (the "Rand" arm of the ablation): offsets uniform in
 * [-h/L, h/L] per axis, weights 1/T, from SplitMix64 seeded with seed. */
void orc_init_rand(int K, int L, int T, uint64_t seed, double *theta) {
  double h = (K - 1) / 2.0, s = h / L;
  uint64_t st = seed;
  for (int j = 0; j < L * T; j++) {
    theta[j * 3 + 0] = (2.0 * orc_uniform(&st) - 1.0) * s;
    theta[j * 3 + 1] = (2.0 * orc_uniform(&st) - 1.0) * s;
    theta[j * 3 + 2] = 1.0 / T;
  }
}

/* ------------------------------------------------------------------------- */
/* Differentiable fit, Eq. 4: Adam (Kingma & Ba 2015; beta1 0.9, beta2 0.999, */
/* eps 1e-8) with the learning rate decayed linearly from lr0 to lr1 over the */
/* steps (Sec. 5.1).  Offsets are optimised in units of the target's half-    */
/* width s = max(1, (K-1)/2) and clamped to |o/s| <= 1 per axis at the start  */
/* and after each step; weights are optimised raw.  init: 0 given (theta_io), 1 radial,      */
/* 2 sparse sampling, 3 random.  loss_hist[steps+1] (if non-NULL) receives    */
/* the loss before every step and after the last.                            */
/* ------------------------------------------------------------------------- */
int orc_fit(const double *tgt, int K, int L, int T, int steps, double lr0,
            double lr1, int init, int loss_kind, double eps, uint64_t seed,
            double *theta_io, double *loss_hist) {
  if (K <= 0 || (K & 1) == 0 || L <= 0 || T <= 0 || steps < 0) return ORC_EINVAL;
  int P = L * T * 3;
  if (init == 1) orc_init_ir(tgt, K, L, T, theta_io);
  else if (init == 2) orc_init_ss(tgt, K, L, T, seed, theta_io);
  else if (init == 3) orc_init_rand(K, L, T, seed, theta_io);
  double s = (K - 1) / 2.0;
  if (s < 1.0) s = 1.0;
  double *m = (double *)calloc(P, sizeof(double)), *v = (double *)calloc(P, sizeof(double));
  double *g = (double *)malloc(sizeof(double) * P), *q = (double *)malloc(sizeof(double) * P);
  /* the canvas bound |o/s| <= 1 holds from the first step, whatever the init */
  for (int j = 0; j < P; j++) {
    q[j] = (j % 3 == 2) ? theta_io[j] : theta_io[j] / s;
    if (j % 3 != 2) { if (q[j] > 1.0) q[j] = 1.0; if (q[j] < -1.0) q[j] = -1.0; }
  }
  const double b1 = 0.9, b2 = 0.999, aeps = 1e-8;
  double b1t = 1.0, b2t = 1.0;
  for (int t = 0; t < steps; t++) {
    for (int j = 0; j < P; j++) theta_io[j] = (j % 3 == 2) ? q[j] : q[j] * s;
    double L0 = orc_fit_loss(theta_io, L, T, tgt, K, loss_kind, eps, g);
    if (loss_hist) loss_hist[t] = L0;
    double lr = steps > 1 ? lr0 + (lr1 - lr0) * (double)t / (double)(steps - 1) : lr0;
    b1t *= b1; b2t *= b2;
    for (int j = 0; j < P; j++) {
      double gj = (j % 3 == 2) ? g[j] : g[j] * s;
      m[j] = b1 * m[j] + (1.0 - b1) * gj;
      v[j] = b2 * v[j] + (1.0 - b2) * gj * gj;
      double mh = m[j] / (1.0 - b1t), vh = v[j] / (1.0 - b2t);
      q[j] -= lr * mh / (sqrt(vh) + aeps);
      if (j % 3 != 2) { if (q[j] > 1.0) q[j] = 1.0; if (q[j] < -1.0) q[j] = -1.0; }
    }
  }
  for (int j = 0; j < P; j++) theta_io[j] = (j % 3 == 2) ? q[j] : q[j] * s;
  if (loss_hist) loss_hist[steps] = orc_fit_loss(theta_io, L, T, tgt, K, loss_kind, eps, NULL);
  free(m); free(v); free(g); free(q);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Dense spatially varying reference (quality reference), Eq. 1 per pixel:    */
/* out[x] = sum_m K_x[m] * I[clamp(x - m)], where K_x = sum_k alpha_k(x) D_k   */
/* blends dense target kernels D_k [B][Kd][Kd] (Kd odd) with the same weights */
/* as Eq. 9.  The x - m indexing makes this a true convolution, which is what */
/* a fitted complex reproduces (its impulse response is its gather stencil    */
/* reflected about the centre).                                               */
/* ------------------------------------------------------------------------- */
int orc_dense_sv(const double *img, int H, int W, int C, const double *maps,
                 int dims, const int *n_nodes, const double *node_vals,
                 const double *lut, int Kd, double *out) {
  if (H <= 0 || W <= 0 || C <= 0 || Kd <= 0 || (Kd & 1) == 0) return ORC_EINVAL;
  int B = dims == 1 ? n_nodes[0] : n_nodes[0] * n_nodes[1];
  int hd = (Kd - 1) / 2;
  long HW = (long)H * W;
#pragma omp parallel
  {
    double *alpha = (double *)malloc(sizeof(double) * B);
    double *ker = (double *)malloc(sizeof(double) * Kd * Kd);
#pragma omp for schedule(static)
    for (long px = 0; px < HW; px++) {
      int v = (int)(px / W), u = (int)(px % W);
      double pv[2] = {maps[px], dims == 2 ? maps[HW + px] : 0.0};
      orc_alpha(pv, dims, n_nodes, node_vals, alpha);
      for (int j = 0; j < Kd * Kd; j++) ker[j] = 0.0;
      for (int k = 0; k < B; k++) {
        if (alpha[k] == 0.0) continue;
        for (int j = 0; j < Kd * Kd; j++) ker[j] += alpha[k] * lut[(long)k * Kd * Kd + j];
      }
      for (int c = 0; c < C; c++) {
        double acc = 0.0;
        for (int my = -hd; my <= hd; my++)
          for (int mx = -hd; mx <= hd; mx++)
            acc += ker[(my + hd) * Kd + (mx + hd)] *
                   fetch(img, H, W, C, v - my, u - mx, c, 0);
        out[px * C + c] = acc;
      }
    }
    free(alpha);
    free(ker);
  }
  return ORC_OK;
}
