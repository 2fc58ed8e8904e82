/*
 * Host renderer of seeded synthetic speckle images (input generation only).
 * Renders any window of an image tile by tile: the pixels' reference-frame
 * coordinates give the cells whose dots can reach the tile, those dots are
 * generated once into a table, and each pixel sums them in the fixed order of
 * syn_speckle_sum. Built with -ffp-contract=off (see speckle.h).
 */
#include <stdlib.h>
#include <string.h>

#include "speckle.h"

#define TILE 32

static int render_tile(const syn_speckle* sp, const syn_field* fd, const syn_intensity* it,
                       int64_t W, int64_t tx0, int64_t ty0, int64_t tw, int64_t th,
                       double* out, int64_t ldo) {
  double X[TILE * TILE], Y[TILE * TILE];
  double xlo = 1e300, xhi = -1e300, ylo = 1e300, yhi = -1e300;
  for (int64_t r = 0; r < th; ++r)
    for (int64_t c = 0; c < tw; ++c) {
      double Xp, Yp;
      syn_inverse_map(fd, (double)(tx0 + c), (double)(ty0 + r), &Xp, &Yp);
      X[r * TILE + c] = Xp;
      Y[r * TILE + c] = Yp;
      if (Xp < xlo) xlo = Xp;
      if (Xp > xhi) xhi = Xp;
      if (Yp < ylo) ylo = Yp;
      if (Yp > yhi) yhi = Yp;
    }
  int64_t i0, i1, j0, j1;
  syn_cell_range(sp, xlo, xhi, ylo, yhi, &i0, &i1, &j0, &j1);
  int64_t ncx = i1 - i0 + 1, ncy = j1 - j0 + 1;
  int kmax = syn_kmax(sp);
  int* counts = (int*)malloc(sizeof(int) * (size_t)(ncx * ncy));
  syn_dotrec* dots = (syn_dotrec*)malloc(sizeof(syn_dotrec) * (size_t)(ncx * ncy * kmax));
  if (!counts || !dots) {
    free(counts);
    free(dots);
    return -1;
  }
  for (int64_t j = j0; j <= j1; ++j)
    for (int64_t i = i0; i <= i1; ++i) {
      int64_t e = (j - j0) * ncx + (i - i0);
      syn_fill_cell(sp, i, j, kmax, &counts[e], &dots[e * kmax]);
    }
  for (int64_t r = 0; r < th; ++r)
    for (int64_t c = 0; c < tw; ++c) {
      double S = syn_speckle_sum_table(sp, counts, dots, kmax, i0, j0, (int)ncx, X[r * TILE + c],
                                       Y[r * TILE + c]);
      out[r * ldo + c] = syn_gray(it, S) + syn_pixel_noise(it, tx0 + c, ty0 + r, W);
    }
  free(counts);
  free(dots);
  return 0;
}

/* Window [x0, x0 + w) x [y0, y0 + h) of a W-wide image into out (h rows of w doubles). */
int syn_render_window(const syn_speckle* sp, const syn_field* fd, const syn_intensity* it,
                      int64_t W, int64_t x0, int64_t y0, int64_t w, int64_t h, double* out) {
  int64_t ntx = (w + TILE - 1) / TILE, nty = (h + TILE - 1) / TILE;
  int err = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : err)
  for (int64_t t = 0; t < ntx * nty; ++t) {
    int64_t bx = t % ntx, by = t / ntx;
    int64_t tx0 = bx * TILE, ty0 = by * TILE;
    int64_t tw = w - tx0 < TILE ? w - tx0 : TILE;
    int64_t th = h - ty0 < TILE ? h - ty0 : TILE;
    err |= render_tile(sp, fd, it, W, x0 + tx0, y0 + ty0, tw, th, out + ty0 * w + tx0, w);
  }
  return err ? -1 : 0;
}

/* Same pixels by the direct per-pixel form (no table); slow, for checking the tiled form. */
int syn_render_window_direct(const syn_speckle* sp, const syn_field* fd, const syn_intensity* it,
                             int64_t W, int64_t x0, int64_t y0, int64_t w, int64_t h,
                             double* out) {
#pragma omp parallel for schedule(dynamic)
  for (int64_t r = 0; r < h; ++r)
    for (int64_t c = 0; c < w; ++c) out[r * w + c] = syn_pixel(sp, fd, it, x0 + c, y0 + r, W);
  return 0;
}

/* Truth: displacement u(X), v(X) at n reference-frame points. */
void syn_displacement_at(const syn_field* fd, const double* X, const double* Y, int64_t n,
                         double* u, double* v) {
  for (int64_t k = 0; k < n; ++k) syn_displacement(fd, X[k], Y[k], &u[k], &v[k]);
}

/* Reference-frame coordinates of n deformed-image points. */
void syn_inverse_map_at(const syn_field* fd, const double* x, const double* y, int64_t n,
                        double* X, double* Y) {
  for (int64_t k = 0; k < n; ++k) syn_inverse_map(fd, x[k], y[k], &X[k], &Y[k]);
}
