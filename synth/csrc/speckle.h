/*
 * Seeded synthetic speckle pairs: a sum of Gaussian dots evaluated at the
 * reference-frame coordinate of each pixel, X = phi^-1(x), for a known
 * displacement field u(X) (x = X + u(X), Lagrangian).
 *
 * This header holds input generation only: no step of the correlation method
 * lives here. It is compiled twice, by gcc for the host renderer and by nvcc
 * for the device renderer, both with floating-point contraction switched off,
 * so that the two produce the same doubles except where libm's exp/log/cos and
 * CUDA's differ by an ulp.
 *
 * Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator: value n of the stream with seed s is mix64(s + (n + 1) * gamma).
 * Dots are stratified: cell (i, j) of side L holds floor(lambda) dots plus one
 * more with probability frac(lambda), lambda = density * L^2, each uniform in
 * its cell, so any window of the image can be rendered from the cells near it.
 */
#ifndef SYNTH_SPECKLE_H
#define SYNTH_SPECKLE_H

#include <math.h>
#include <stdint.h>

#ifdef __CUDACC__
#define SYN_HD __host__ __device__ __forceinline__
#else
#define SYN_HD static inline
#endif

#define SYN_GAMMA 0x9E3779B97F4A7C15ULL
#define SYN_CELL_BIAS 1048576LL /* 2^20: cell indices may be negative */
#define SYN_MAX_PER_CELL 62

typedef struct {
  uint64_t seed;
  double density;   /* dots per px^2 */
  double sigma_lo;  /* dot radius sigma, uniform in [lo, hi) */
  double sigma_hi;
  double amp_lo;    /* dot amplitude, uniform in [lo, hi) */
  double amp_hi;
  double cutoff;    /* a dot contributes where its distance is < cutoff */
  int32_t cell;     /* stratification cell side L in px */
  int32_t pad_;
} syn_speckle;

enum { SYN_FIELD_IDENTITY = 0, SYN_FIELD_AFFINE = 1, SYN_FIELD_SINE_V = 2, SYN_FIELD_QUADRATIC = 3 };

typedef struct {
  int32_t kind;
  int32_t pad_;
  double cx, cy;          /* origin of the centred coordinates (X', Y') */
  /* affine: u = u0 + exx X' + exy Y', v = v0 + eyx X' + eyy Y' */
  double u0, v0, exx, exy, eyx, eyy;
  /* extra rigid slip of `jump` px along (1,1)/sqrt(2) where Y' > X' */
  double jump;
  /* sine: u = 0, v = amp sin(2 pi Y / T(X)), T = t0 + (t1 - t0) X / (W - 1),
     X, Y plain pixel coordinates */
  double amp, t0, t1;
  double width;           /* W used by T(X) */
  /* quadratic: the affine terms plus u += uxx X'^2 + uxy X'Y' + uyy Y'^2, v likewise */
  double uxx, uxy, uyy, vxx, vxy, vyy;
} syn_field;

typedef struct {
  double gray_max;   /* G: 255, 4095, 65535 or 1.0 */
  double noise;      /* additive Gaussian noise sigma, in gray levels */
  uint64_t noise_seed;
} syn_intensity;

SYN_HD uint64_t syn_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

SYN_HD uint64_t syn_splitmix(uint64_t seed, uint64_t n) {
  return syn_mix64(seed + (n + 1ULL) * SYN_GAMMA);
}

/* uniform double in [0, 1) with 53 random bits */
SYN_HD double syn_u01(uint64_t seed, uint64_t n) {
  return (double)(syn_splitmix(seed, n) >> 11) * (1.0 / 9007199254740992.0);
}

SYN_HD uint64_t syn_cell_id(int64_t i, int64_t j) {
  return (uint64_t)(i + SYN_CELL_BIAS) * 2097152ULL + (uint64_t)(j + SYN_CELL_BIAS);
}

/* counter of field f (0..7) of dot k (0..63) in cell id */
SYN_HD uint64_t syn_counter(uint64_t id, int k, int f) {
  return ((id * 64ULL + (uint64_t)k) * 8ULL) + (uint64_t)f;
}

SYN_HD int syn_cell_count(const syn_speckle* sp, int64_t i, int64_t j) {
  double lam = sp->density * (double)sp->cell * (double)sp->cell;
  int base = (int)floor(lam);
  double frac = lam - (double)base;
  int n = base + (syn_u01(sp->seed, syn_counter(syn_cell_id(i, j), 63, 7)) < frac ? 1 : 0);
  return n > SYN_MAX_PER_CELL ? SYN_MAX_PER_CELL : n;
}

/* dot k of cell (i, j): centre (px, py), sigma s, amplitude a */
SYN_HD void syn_dot(const syn_speckle* sp, int64_t i, int64_t j, int k, double* px, double* py,
                    double* s, double* a) {
  uint64_t id = syn_cell_id(i, j);
  double L = (double)sp->cell;
  *px = ((double)i + syn_u01(sp->seed, syn_counter(id, k, 0))) * L;
  *py = ((double)j + syn_u01(sp->seed, syn_counter(id, k, 1))) * L;
  *s = sp->sigma_lo + (sp->sigma_hi - sp->sigma_lo) * syn_u01(sp->seed, syn_counter(id, k, 2));
  *a = sp->amp_lo + (sp->amp_hi - sp->amp_lo) * syn_u01(sp->seed, syn_counter(id, k, 3));
}

/* one dot's contribution at (X, Y); zero beyond the cutoff radius */
SYN_HD double syn_dot_value(double X, double Y, double px, double py, double s, double a,
                            double cutoff) {
  double ddx = X - px;
  double ddy = Y - py;
  double d2 = ddx * ddx + ddy * ddy;
  if (d2 >= cutoff * cutoff) return 0.0;
  return a * exp(-d2 / (2.0 * s * s));
}

/* S(X): cells are visited row by row (j outer, i inner), dots in order k */
SYN_HD double syn_speckle_sum(const syn_speckle* sp, double X, double Y) {
  double L = (double)sp->cell;
  int64_t i0 = (int64_t)floor((X - sp->cutoff) / L);
  int64_t i1 = (int64_t)floor((X + sp->cutoff) / L);
  int64_t j0 = (int64_t)floor((Y - sp->cutoff) / L);
  int64_t j1 = (int64_t)floor((Y + sp->cutoff) / L);
  double acc = 0.0;
  for (int64_t j = j0; j <= j1; ++j)
    for (int64_t i = i0; i <= i1; ++i) {
      int n = syn_cell_count(sp, i, j);
      for (int k = 0; k < n; ++k) {
        double px, py, s, a;
        syn_dot(sp, i, j, k, &px, &py, &s, &a);
        acc += syn_dot_value(X, Y, px, py, s, a, sp->cutoff);
      }
    }
  return acc;
}

/* one generated dot, as held in a tile's table */
typedef struct {
  double px, py, s, a;
} syn_dotrec;

SYN_HD int syn_kmax(const syn_speckle* sp) {
  double lam = sp->density * (double)sp->cell * (double)sp->cell;
  int k = (int)floor(lam) + 1;
  return k > SYN_MAX_PER_CELL ? SYN_MAX_PER_CELL : k;
}

/* cell range [i0, i1] x [j0, j1] that S(X) visits for X in [xlo, xhi] x [ylo, yhi] */
SYN_HD void syn_cell_range(const syn_speckle* sp, double xlo, double xhi, double ylo, double yhi,
                           int64_t* i0, int64_t* i1, int64_t* j0, int64_t* j1) {
  double L = (double)sp->cell;
  *i0 = (int64_t)floor((xlo - sp->cutoff) / L);
  *i1 = (int64_t)floor((xhi + sp->cutoff) / L);
  *j0 = (int64_t)floor((ylo - sp->cutoff) / L);
  *j1 = (int64_t)floor((yhi + sp->cutoff) / L);
}

/* entry e = (j - cj0) * ncx + (i - ci0) of a table holding cells from (ci0, cj0) */
SYN_HD void syn_fill_cell(const syn_speckle* sp, int64_t i, int64_t j, int kmax, int* count,
                          syn_dotrec* dots) {
  int n = syn_cell_count(sp, i, j);
  *count = n;
  for (int k = 0; k < n && k < kmax; ++k)
    syn_dot(sp, i, j, k, &dots[k].px, &dots[k].py, &dots[k].s, &dots[k].a);
}

/* S(X) from a table; visits cells and dots in the same order as syn_speckle_sum */
SYN_HD double syn_speckle_sum_table(const syn_speckle* sp, const int* counts,
                                    const syn_dotrec* dots, int kmax, int64_t ci0, int64_t cj0,
                                    int ncx, double X, double Y) {
  int64_t i0, i1, j0, j1;
  syn_cell_range(sp, X, X, Y, Y, &i0, &i1, &j0, &j1);
  double acc = 0.0;
  for (int64_t j = j0; j <= j1; ++j)
    for (int64_t i = i0; i <= i1; ++i) {
      int64_t e = (j - cj0) * ncx + (i - ci0);
      int n = counts[e];
      const syn_dotrec* d = dots + e * kmax;
      for (int k = 0; k < n; ++k) acc += syn_dot_value(X, Y, d[k].px, d[k].py, d[k].s, d[k].a, sp->cutoff);
    }
  return acc;
}

/* gray level from S, before noise */
SYN_HD double syn_gray(const syn_intensity* it, double S) {
  return it->gray_max * (0.1 + 0.8 * (1.0 - exp(-S)));
}

/* Reference-frame coordinate X of deformed-image pixel x (x = X + u(X)). */
SYN_HD void syn_inverse_map(const syn_field* fd, double x, double y, double* X, double* Y) {
  if (fd->kind == SYN_FIELD_AFFINE) {
    double a = 1.0 + fd->exx, b = fd->exy, c = fd->eyx, d = 1.0 + fd->eyy;
    double det = a * d - b * c;
    double rx = x - fd->cx, ry = y - fd->cy;
    /* without the slip */
    double qx = rx - fd->u0, qy = ry - fd->v0;
    double Xa = (d * qx - b * qy) / det;
    double Ya = (-c * qx + a * qy) / det;
    if (fd->jump != 0.0) {
      double jx = fd->jump * 0.70710678118654752440, jy = jx;
      double sx = qx - jx, sy = qy - jy;
      double Xb = (d * sx - b * sy) / det;
      double Yb = (-c * sx + a * sy) / det;
      if (Yb > Xb) { Xa = Xb; Ya = Yb; }
    }
    *X = Xa + fd->cx;
    *Y = Ya + fd->cy;
    return;
  }
  if (fd->kind == SYN_FIELD_QUADRATIC) {
    /* Newton's method on X + u(X) = x from X = x */
    double Xc = x - fd->cx, Yc = y - fd->cy;
    double rx0 = Xc, ry0 = Yc;
    for (int itn = 0; itn < 100; ++itn) {
      double fu = fd->u0 + fd->exx * Xc + fd->exy * Yc + fd->uxx * Xc * Xc + fd->uxy * Xc * Yc +
                  fd->uyy * Yc * Yc;
      double fv = fd->v0 + fd->eyx * Xc + fd->eyy * Yc + fd->vxx * Xc * Xc + fd->vxy * Xc * Yc +
                  fd->vyy * Yc * Yc;
      double rx = Xc + fu - rx0, ry = Yc + fv - ry0;
      double a = 1.0 + fd->exx + 2.0 * fd->uxx * Xc + fd->uxy * Yc;
      double b = fd->exy + fd->uxy * Xc + 2.0 * fd->uyy * Yc;
      double c = fd->eyx + 2.0 * fd->vxx * Xc + fd->vxy * Yc;
      double d = 1.0 + fd->eyy + fd->vxy * Xc + 2.0 * fd->vyy * Yc;
      double det = a * d - b * c;
      double sx = (d * rx - b * ry) / det, sy = (-c * rx + a * ry) / det;
      Xc -= sx;
      Yc -= sy;
      if (fabs(sx) < 1e-13 && fabs(sy) < 1e-13) break;
    }
    *X = Xc + fd->cx;
    *Y = Yc + fd->cy;
    return;
  }
  if (fd->kind == SYN_FIELD_SINE_V) {
    /* u = 0 so X = x; Y solves Y + amp sin(2 pi Y / T(x)) = y, by fixed point */
    double T = fd->t0 + (fd->t1 - fd->t0) * x / (fd->width - 1.0);
    double w = 6.283185307179586476925 / T;
    double Yk = y;
    for (int it = 0; it < 200; ++it) {
      double Yn = y - fd->amp * sin(w * Yk);
      double dlt = Yn - Yk;
      Yk = Yn;
      if (dlt < 1e-13 && dlt > -1e-13) break;
    }
    *X = x;
    *Y = Yk;
    return;
  }
  *X = x;
  *Y = y;
}

/* forward displacement u(X) at reference coordinate X (the truth) */
SYN_HD void syn_displacement(const syn_field* fd, double X, double Y, double* u, double* v) {
  if (fd->kind == SYN_FIELD_QUADRATIC) {
    double Xc = X - fd->cx, Yc = Y - fd->cy;
    *u = fd->u0 + fd->exx * Xc + fd->exy * Yc + fd->uxx * Xc * Xc + fd->uxy * Xc * Yc +
         fd->uyy * Yc * Yc;
    *v = fd->v0 + fd->eyx * Xc + fd->eyy * Yc + fd->vxx * Xc * Xc + fd->vxy * Xc * Yc +
         fd->vyy * Yc * Yc;
    return;
  }
  if (fd->kind == SYN_FIELD_AFFINE) {
    double Xc = X - fd->cx, Yc = Y - fd->cy;
    *u = fd->u0 + fd->exx * Xc + fd->exy * Yc;
    *v = fd->v0 + fd->eyx * Xc + fd->eyy * Yc;
    if (fd->jump != 0.0 && Yc > Xc) {
      *u += fd->jump * 0.70710678118654752440;
      *v += fd->jump * 0.70710678118654752440;
    }
    return;
  }
  if (fd->kind == SYN_FIELD_SINE_V) {
    double T = fd->t0 + (fd->t1 - fd->t0) * X / (fd->width - 1.0);
    *u = 0.0;
    *v = fd->amp * sin(6.283185307179586476925 * Y / T);
    return;
  }
  *u = 0.0;
  *v = 0.0;
}

/* standard normal from two uniforms (Box & Muller 1958) */
SYN_HD double syn_normal(uint64_t seed, uint64_t n) {
  double u1 = 1.0 - syn_u01(seed, 2ULL * n);
  double u2 = syn_u01(seed, 2ULL * n + 1ULL);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}

/* noise sample added to pixel (x, y) of a W-wide image */
SYN_HD double syn_pixel_noise(const syn_intensity* it, int64_t x, int64_t y, int64_t W) {
  if (it->noise > 0.0) return it->noise * syn_normal(it->noise_seed, (uint64_t)(y * W + x));
  return 0.0;
}

/* gray level of pixel (x, y) of a W-wide image, before quantisation (direct form) */
SYN_HD double syn_pixel(const syn_speckle* sp, const syn_field* fd, const syn_intensity* it,
                        int64_t x, int64_t y, int64_t W) {
  double X, Y;
  syn_inverse_map(fd, (double)x, (double)y, &X, &Y);
  return syn_gray(it, syn_speckle_sum(sp, X, Y)) + syn_pixel_noise(it, x, y, W);
}

/* round half to even, then clip to [0, G] */
SYN_HD double syn_quantise(double v, double G) {
  double r = rint(v);
  if (r < 0.0) r = 0.0;
  if (r > G) r = G;
  return r;
}

#endif
