// The wave kernel (template) and its launch helpers, shared by the translation
// units that instantiate it (wave_inst_*.cu); correlate.cu holds the dispatch.
//
// One propagation wave: every point on the frontier is correlated by one block.
//
// Per point (Sec. 2.2, Eq. 4, Eq. 5; Sec. 2.4 for the propagation):
//   1. starting warp: the seed's integer offset (wave 0), else the warp of the
//      accepted 4-neighbour with the highest ZNCC, re-expanded about this centre;
//   2. reference subset: f, f - f_m and the exact gradient of the reference
//      interpolant (cubic B-spline, or bicubic convolution) at the S x S pixels,
//      and the Gauss-Newton Hessian
//      H = sum SD^T SD of the steepest-descent images SD = grad f . dxi/dp,
//      assembled from gradient moments; its Jacobi-scaled inverse by warp-parallel
//      Gauss-Jordan (FP32 on the mixed path, with an FP64 fallback; FP64 on the
//      FP64 path);
//   3. inverse-compositional Gauss-Newton (or Levenberg-Marquardt): sample the
//      deformed interpolant at the warped pixels, reduce sum g, sum g^2, sum SD g
//      and sum f g, solve dp = -H^-1 b with b = sum SD e of the cost (Eq. 2-4),
//      update p <- p o dp^-1, stop when ||dp|| < threshold;
//   4. ZNCC = sum (f - f_m)(g - g_m) / (df dg) from the converging iteration's
//      sampling pass (Levenberg-Marquardt: one more pass at the final p); accept
//      when converged, in bounds and ZNCC >= cut-off;
//   5. an accepted point claims its unvisited in-ROI 4-neighbours for the next wave.
//
// Threads map to pixels by column: thread t < S * bands owns column t % S and
// the rows of band t / S. The deformed coefficients around the warped subset are
// staged in shared memory once and re-staged only when the subset leaves them.
#pragma once

#include <math.h>

#include <type_traits>

#include "dic_internal.cuh"
#include "tma.cuh"

namespace dic {
namespace {

template <int NP>
struct Shape;
template <>
struct Shape<2> { static constexpr int D = 0; };
template <>
struct Shape<6> { static constexpr int D = 1; };
template <>
struct Shape<12> { static constexpr int D = 2; };

// Steepest-descent component c (Eq. 5 Jacobian at p = 0) is
//   (t ? fy : fx) * dx^i * dy^j  with (t, i, j) below.
__host__ __device__ constexpr int sd_t(int c) {
  return (c == 1 || c == 4 || c == 5 || c >= 9) ? 1 : 0;
}
__host__ __device__ constexpr int sd_i(int c) {
  return (c == 2 || c == 4 || c == 7 || c == 10) ? 1 : (c == 6 || c == 9) ? 2 : 0;
}
__host__ __device__ constexpr int sd_j(int c) {
  return (c == 3 || c == 5 || c == 7 || c == 10) ? 1 : (c == 8 || c == 11) ? 2 : 0;
}
// packed index of monomial dx^i dy^j, i + j <= M
__host__ __device__ constexpr int mono(int i, int j, int M) { return j * (M + 1) - j * (j - 1) / 2 + i; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// barrier id among the first `count` threads of the block (id 0 is __syncthreads)
__device__ __forceinline__ void named_barrier_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Warp sums of K values per thread (K a power of two, <= 32) in K - 1 + 5 - log2 K
// shuffles: each step sends half of the remaining values to the partner lane and
// keeps the other half, so lane l ends with the warp sum of v[l >> (5 - log2 K)].
template <typename T, int K>
__device__ __forceinline__ T warp_transpose_sum(T (&v)[K], int lane) {
  int o = 16;
#pragma unroll
  for (int h = K / 2; h >= 1; h >>= 1, o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const T send = upper ? v[i] : v[i + h];
      const T keep = upper ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  T s = v[0];
#pragma unroll
  for (; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

__host__ __device__ constexpr int pow2ceil(int n) {
  int k = 1;
  while (k < n) k <<= 1;
  return k;
}

template <int K>
struct Log2 {
  static constexpr int kValue = K <= 1 ? 0 : 1 + Log2<K / 2>::kValue;
};
template <>
struct Log2<1> {
  static constexpr int kValue = 0;
};

// p <- W(W^-1(.; dp); p) for the quadratic warp, through the second-order
// monomial map m(W(x; p)) ~= A(p) m(x), m = [x^2, xy, y^2, x, y, 1] (terms above
// second order dropped): the new x' and y' rows are Z = R A(dp)^-1 with R the x',
// y' rows of A(p). Write A(dp) = [[I + E, e], [0, 1]] (E: 5 x 5, formed without
// its identity part; e: the constant column) and R = [r, p0|p1]. Then
// Z[:, 0:5] = r + delta with delta (I + E) = -r E, and Z[:, 5] = R[:, 5] - Z[:, 0:5] e.
// Only the increments delta are solved for, so p keeps the full precision of C;
// I + E is near the identity for any increment the iteration takes, so the
// elimination runs without row exchanges, in registers.
template <typename C>
__device__ __forceinline__ void compose_quadratic(C* p, const C* dp) {
  const C u = dp[0], v = dp[1], e2 = dp[2], b = dp[3], c = dp[4], e5 = dp[5];
  const C a = C(1) + e2, d = C(1) + e5;
  const C q6 = dp[6], q7 = dp[7], q8 = dp[8], q9 = dp[9], q10 = dp[10], q11 = dp[11];
  C E[5][5];
  // x'^2 row
  E[0][0] = e2 * (C(2) + e2) + C(2) * u * q6;
  E[0][1] = C(2) * a * b + C(2) * u * q7;
  E[0][2] = b * b + C(2) * u * q8;
  E[0][3] = C(2) * u * a;
  E[0][4] = C(2) * u * b;
  // x'y' row
  E[1][0] = a * c + u * q9 + v * q6;
  E[1][1] = e2 + e5 + e2 * e5 + b * c + u * q10 + v * q7;
  E[1][2] = b * d + u * q11 + v * q8;
  E[1][3] = u * c + v * a;
  E[1][4] = u * d + v * b;
  // y'^2 row
  E[2][0] = c * c + C(2) * v * q9;
  E[2][1] = C(2) * c * d + C(2) * v * q10;
  E[2][2] = e5 * (C(2) + e5) + C(2) * v * q11;
  E[2][3] = C(2) * v * c;
  E[2][4] = C(2) * v * d;
  // x', y' rows
  E[3][0] = q6; E[3][1] = q7; E[3][2] = q8; E[3][3] = e2; E[3][4] = b;
  E[4][0] = q9; E[4][1] = q10; E[4][2] = q11; E[4][3] = c; E[4][4] = e5;
  const C ec[5] = {u * u, u * v, v * v, u, v};
  // right-hand sides -r E, with r = [p6, p7, p8, 1 + p2, p3] and [p9, p10, p11, p4, 1 + p5]
  C d0[5], d1[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    d0[j] = -(E[3][j] + (p[2] * E[3][j] + p[6] * E[0][j] + p[7] * E[1][j] + p[8] * E[2][j] + p[3] * E[4][j]));
    d1[j] = -(E[4][j] + (p[5] * E[4][j] + p[9] * E[0][j] + p[10] * E[1][j] + p[11] * E[2][j] + p[4] * E[3][j]));
  }
  // delta (I + E) = rhs  <=>  (I + E)^T delta^T = rhs^T: elimination on T = (I + E)^T
  C T[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) T[i][j] = (i == j ? C(1) : C(0)) + E[j][i];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const C inv = C(1) / T[k][k];
#pragma unroll
    for (int i = k + 1; i < 5; ++i) {
      const C f = T[i][k] * inv;
#pragma unroll
      for (int j = k + 1; j < 5; ++j) T[i][j] -= f * T[k][j];
      d0[i] -= f * d0[k];
      d1[i] -= f * d1[k];
    }
    T[k][k] = inv;
  }
#pragma unroll
  for (int i = 4; i >= 0; --i) {
    C s0 = d0[i], s1 = d1[i];
#pragma unroll
    for (int j = i + 1; j < 5; ++j) {
      s0 -= T[i][j] * d0[j];
      s1 -= T[i][j] * d1[j];
    }
    d0[i] = s0 * T[i][i];
    d1[i] = s1 * T[i][i];
  }
  const C n0 = p[0] - (ec[3] * (C(1) + p[2] + d0[3]) + ec[4] * (p[3] + d0[4]) + ec[0] * (p[6] + d0[0]) +
                       ec[1] * (p[7] + d0[1]) + ec[2] * (p[8] + d0[2]));
  const C n1 = p[1] - (ec[3] * (p[4] + d1[3]) + ec[4] * (C(1) + p[5] + d1[4]) + ec[0] * (p[9] + d1[0]) +
                       ec[1] * (p[10] + d1[1]) + ec[2] * (p[11] + d1[2]));
  p[0] = n0;
  p[1] = n1;
  p[2] += d0[3];
  p[3] += d0[4];
  p[4] += d1[3];
  p[5] += d1[4];
  p[6] += d0[0];
  p[7] += d0[1];
  p[8] += d0[2];
  p[9] += d1[0];
  p[10] += d1[1];
  p[11] += d1[2];
}

// p <- W(W^-1(.; dp); p) in the working precision C. Rigid: p - dp. Affine, exact:
// with A = I + [[p2, p3], [p4, p5]], F = [[dp2, dp3], [dp4, dp5]] and
// E = (I + F)^-1 - I = -(I + F)^-1 F, the new linear part is A + A E and the new
// translation t - (A + A E) dt; only the small increments A E and -(A + A E) dt
// are formed, so p keeps the full precision of C. Quadratic: compose_quadratic in C.
template <typename C, int NP>
__device__ void compose_inverse(C* p, const C* dp) {
  if (NP == 2) {
    p[0] -= dp[0];
    p[1] -= dp[1];
  } else if (NP == 6) {
    const C d2 = dp[2], d3 = dp[3], d4 = dp[4], d5 = dp[5];
    const C inv = C(1) / ((C(1) + d2) * (C(1) + d5) - d3 * d4);
    const C i00 = (C(1) + d5) * inv, i01 = -d3 * inv, i10 = -d4 * inv, i11 = (C(1) + d2) * inv;
    const C e00 = -(i00 * d2 + i01 * d4), e01 = -(i00 * d3 + i01 * d5);
    const C e10 = -(i10 * d2 + i11 * d4), e11 = -(i10 * d3 + i11 * d5);
    const C a00 = C(1) + p[2], a01 = p[3], a10 = p[4], a11 = C(1) + p[5];
    const C g00 = a00 * e00 + a01 * e10, g01 = a00 * e01 + a01 * e11;
    const C g10 = a10 * e00 + a11 * e10, g11 = a10 * e01 + a11 * e11;
    const C n00 = a00 + g00, n01 = a01 + g01, n10 = a10 + g10, n11 = a11 + g11;
    p[0] -= n00 * dp[0] + n01 * dp[1];
    p[1] -= n10 * dp[0] + n11 * dp[1];
    p[2] += g00;
    p[3] += g01;
    p[4] += g10;
    p[5] += g11;
  } else {
    compose_quadratic<C>(p, dp);
  }
}

// neighbour warp re-expanded about a centre offset (ddx, ddy) from it
template <typename C, int NP>
__device__ void transfer_warp(const C* pn, C ddx, C ddy, C* p) {
  for (int c = 0; c < NP; ++c) p[c] = pn[c];
  if (NP >= 6) {
    p[0] = pn[0] + pn[2] * ddx + pn[3] * ddy;
    p[1] = pn[1] + pn[4] * ddx + pn[5] * ddy;
  }
  if (NP >= 12) {
    p[0] += pn[6] * ddx * ddx + pn[7] * ddx * ddy + pn[8] * ddy * ddy;
    p[1] += pn[9] * ddx * ddx + pn[10] * ddx * ddy + pn[11] * ddy * ddy;
    p[2] = pn[2] + C(2) * pn[6] * ddx + pn[7] * ddy;
    p[3] = pn[3] + pn[7] * ddx + C(2) * pn[8] * ddy;
    p[4] = pn[4] + C(2) * pn[9] * ddx + pn[10] * ddy;
    p[5] = pn[5] + pn[10] * ddx + C(2) * pn[11] * ddy;
  }
}

template <typename C>
__device__ __forceinline__ bool is_flat(C delta, C mean, int count) {
  return delta / sqrt(static_cast<C>(count)) <= C(1e-6) * fmax(fabs(mean), C(1));
}

// n < 2^23 as a float, exactly, on the integer and FP32 pipes (0x4B000000 | n is the
// float 2^23 + n)
__device__ __forceinline__ float small_uint_to_float(uint32_t n) {
  return __uint_as_float(0x4B000000u | n) - 8388608.0f;
}

// Gray level at subset column c, row r of a staged gray tile (row pitch in bytes).
template <typename T>
__device__ __forceinline__ T tile_gray(const unsigned char* tile, int pitch, int dtype, int c, int r) {
  const unsigned char* row = tile + r * pitch;
  switch (dtype) {
    case DIC_U8:
      if constexpr (sizeof(T) == sizeof(float)) return small_uint_to_float(row[c]);
      return static_cast<T>(row[c]);
    case DIC_U16:
      if constexpr (sizeof(T) == sizeof(float))
        return small_uint_to_float(reinterpret_cast<const uint16_t*>(row)[c]);
      return static_cast<T>(reinterpret_cast<const uint16_t*>(row)[c]);
    case DIC_BF16:
      return static_cast<T>(__uint_as_float(static_cast<uint32_t>(reinterpret_cast<const uint16_t*>(row)[c]) << 16));
    case DIC_F32:
      return static_cast<T>(reinterpret_cast<const float*>(row)[c]);
    default:
      return static_cast<T>(reinterpret_cast<const double*>(row)[c]);
  }
}

struct Window {
  int x0, y0, w, h;   // origin in the image, row pitch and rows in shared memory
};

// Solve state. FP64 path: the Hessian, its inverse and the vectors of the
// refined FP64 solve. Mixed path: the inverse only, in FP32, stored by columns
// (element (i, j) at j NP + i) so that lane i reads row i without bank conflicts.
template <typename C, int NP>
struct SolveState;
template <int NP>
struct SolveState<double, NP> {
  double H[NP * NP];        // Gauss-Newton Hessian
  double X[NP * NP];        // its inverse
  double bvec[NP];          // right-hand side, then the residual
  double dvec[NP];          // first solution
};
template <int NP>
struct SolveState<float, NP> {
  float X[NP * NP];         // H^-1 = D (D H D)^-1 D, column-major
};
// FP64 solves on the FP32 path (kernel variant 3): the FP64 Hessian and the FP32
// inverse of the mixed path, which preconditions an FP64 iterative refinement
struct Refined64 {};
template <int NP>
struct SolveState<Refined64, NP> {
  float X[NP * NP];         // H^-1 = D (D H D)^-1 D in FP32, column-major
  double H[NP * NP];        // Gauss-Newton Hessian in FP64 (from the FP32 moment sums)
};

// Per-block state of the point being correlated; C is the working precision
// (float on the mixed path, double on the FP64 path), SC the precision of the
// Hessian inverse and the solve (C, or Refined64 on the mixed path with FP64 solves).
template <typename C, int NP, typename SC = C>
struct PointState {
  SolveState<SC, NP> sv;
  C p[kMaxParams];          // current warp
  C dp[kMaxParams];         // last update
  C sdf[NP];                // sum SD (f - f_m)
  C sds[NP];                // sum SD
  C mu;                     // mean of f' = f - f0 (f0: reference gray level at the centre)
  C delta_f;                // ||f - f_m||
  C sf, sff;                // sum f', sum f'^2 (the NSSD norm ||f||)
  C f0;
  double mu64, delta_f64;   // mean and contrast of f' in FP64 (mixed path with FP64 solves)
  double zncc;
  int q, item, ctl, iters, status, converged, stage;
  int inside;               // every sample of the next pass lies inside the sampling bounds
  Window win, next;
};

// Warp-parallel Gauss-Jordan inverse of the SPD matrix H (row-major, N x N) in the
// precision V: lane j < N carries column j of H, lane N + j column j of the
// identity. No row exchanges: the pivots of an SPD matrix are positive and equal
// the LDL^T pivots. Returns the smallest pivot divided by the largest diagonal
// entry (<= 0 when a pivot is not positive); X receives the inverse.
template <typename V, int N>
__device__ double invert_spd_warp(const double* H, double* X, int lane) {
  V col[N];
  const bool mine = lane < 2 * N;
#pragma unroll
  for (int i = 0; i < N; ++i)
    col[i] = !mine ? V(0) : (lane < N ? static_cast<V>(H[i * N + lane]) : (i == lane - N ? V(1) : V(0)));
  double dmax = 0.0;
#pragma unroll
  for (int k = 0; k < N; ++k) dmax = fmax(dmax, fabs(H[k * N + k]));
  V pmin = V(1e30);
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const V piv = __shfl_sync(0xffffffffu, col[k], k);
    pmin = piv < pmin ? piv : pmin;
    if (!(piv > V(0))) return 0.0;
    col[k] = col[k] / piv;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (i == k) continue;
      const V f = __shfl_sync(0xffffffffu, col[i], k);
      col[i] -= f * col[k];
    }
  }
  if (mine && lane >= N) {
#pragma unroll
    for (int i = 0; i < N; ++i) X[i * N + (lane - N)] = static_cast<double>(col[i]);
  }
  return dmax > 0.0 ? static_cast<double>(pmin) / dmax : 0.0;
}

// Warp-parallel Gauss-Jordan inverse of the Jacobi-scaled SPD matrix D H D,
// D = diag(H_ii^-1/2), in the precision V: lane j < N carries column j of D H D,
// lane N + j column j of the identity; no row exchanges (SPD). H(i, j) comes from
// hget. The unit diagonal removes the spread of the monomial scales (up to r^4
// between the translation and quadratic columns), so FP32 suffices unless H itself
// is ill-conditioned. Writes H^-1 = D (D H D)^-1 D column-major into X. Returns
// the smallest scaled pivot; *ratio receives the smallest pivot of H itself (the
// scaled pivot k times H_kk) over the largest diagonal entry (0 when a pivot is
// not positive).
template <typename V, int N, typename HGet>
__device__ __forceinline__ float invert_scaled_warp(HGet hget, float* X, int lane, float* ratio) {
  // lane i < N: d_i = H_ii^-1/2 (shared by shuffles)
  const V hii = lane < N ? static_cast<V>(hget(lane, lane)) : V(0);
  V dl = V(0);
  if constexpr (sizeof(V) == sizeof(float)) {
    dl = hii > V(0) ? rsqrtf(hii) : V(0);
  } else {
    dl = hii > V(0) ? V(1) / sqrt(hii) : V(0);
  }
  V hmax = hii;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const V t = __shfl_xor_sync(0xffffffffu, hmax, o);
    hmax = t > hmax ? t : hmax;
  }
  const bool mine = lane < 2 * N;
  const int j = lane < N ? lane : (lane < 2 * N ? lane - N : 0);
  const V dj = __shfl_sync(0xffffffffu, dl, j);
  V col[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const V di = __shfl_sync(0xffffffffu, dl, i);
    col[i] = !mine ? V(0) : (lane < N ? static_cast<V>(hget(i, j)) * di * dj : (i == j ? V(1) : V(0)));
  }
  V pmin = V(1e30), rmin = V(1e30);
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const V piv = __shfl_sync(0xffffffffu, col[k], k);
    const V hkk = __shfl_sync(0xffffffffu, hii, k);
    pmin = piv < pmin ? piv : pmin;
    const V up = piv * hkk;   // the pivot of H itself: the scaled pivot times H_kk
    rmin = up < rmin ? up : rmin;
    if (!(piv > V(0))) {
      *ratio = 0.0f;
      return 0.0f;
    }
    if constexpr (sizeof(V) == sizeof(float))
      col[k] *= __frcp_rn(piv);
    else
      col[k] *= V(1) / piv;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (i == k) continue;
      const V f = __shfl_sync(0xffffffffu, col[i], k);
      col[i] -= f * col[k];
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const V di = __shfl_sync(0xffffffffu, dl, i);
    if (mine && lane >= N) X[j * N + i] = static_cast<float>(col[i] * di * dj);
  }
  *ratio = hmax > V(0) ? static_cast<float>(rmin / hmax) : 0.0f;
  return static_cast<float>(pmin);
}

// The FP64 fallback of invert_scaled_warp, out of line to keep its registers
// away from the rest of the kernel; H is read from the FP32 moment sums.
template <int N, int NMOM, int M2>
__device__ __noinline__ void invert_scaled_fp64(const float* out, float* X, int lane, float* ratio) {
  auto hget = [&](int ca, int cb) -> float {
    return out[(sd_t(ca) + sd_t(cb)) * NMOM + mono(sd_i(ca) + sd_i(cb), sd_j(ca) + sd_j(cb), M2)];
  };
  invert_scaled_warp<double, N>(hget, X, lane, ratio);
}

// Coefficients under the warped subset: [x0, x1] x [y0, y1] holds the 4 x 4 support of
// every sample, from a bound on the warped offsets (0.05 px slack covers the
// evaluation of the positions), clamped to the image. *inside: every sample position
// lies in the sampling bounds 1 <= x < W - 2, 1 <= y < H - 2 (then the per-sample
// test can be skipped). False for a non-finite or absurd warp, or when nothing of
// the support lies in the image.
template <typename C, int NP>
__device__ bool needed_range(const C* p, int xc, int yc, int r, int W, int H, int* x0, int* x1, int* y0,
                             int* y1, int* inside) {
  float ex, ey;
  const float rf = static_cast<float>(r);
  const float q0 = static_cast<float>(p[0]), q1 = static_cast<float>(p[1]);
  if (NP >= 6) {
    ex = rf * (fabsf(1.0f + static_cast<float>(p[2])) + fabsf(static_cast<float>(p[3])));
    ey = rf * (fabsf(static_cast<float>(p[4])) + fabsf(1.0f + static_cast<float>(p[5])));
  } else {
    ex = ey = rf;
  }
  if (NP >= 12) {
    ex += rf * rf * (fabsf(static_cast<float>(p[6])) + fabsf(static_cast<float>(p[7])) +
                     fabsf(static_cast<float>(p[8])));
    ey += rf * rf * (fabsf(static_cast<float>(p[9])) + fabsf(static_cast<float>(p[10])) +
                     fabsf(static_cast<float>(p[11])));
  }
  ex += 0.05f;
  ey += 0.05f;
  if (!(fabsf(q0) < 1e6f && fabsf(q1) < 1e6f && ex < 1e6f && ey < 1e6f)) return false;
  *inside = static_cast<float>(xc) + q0 - ex >= 1.0f && static_cast<float>(xc) + q0 + ex < static_cast<float>(W - 2) &&
            static_cast<float>(yc) + q1 - ey >= 1.0f && static_cast<float>(yc) + q1 + ey < static_cast<float>(H - 2);
  *x0 = max(xc + static_cast<int>(floorf(q0 - ex)) - 1, 0);
  *x1 = min(xc + static_cast<int>(floorf(q0 + ex)) + 2, W - 1);
  *y0 = max(yc + static_cast<int>(floorf(q1 - ey)) - 1, 0);
  *y1 = min(yc + static_cast<int>(floorf(q1 + ey)) + 2, H - 1);
  return *x1 >= *x0 && *y1 >= *y0;
}

// Lane 0: the window for sampling at st.p. stage 0: the staged window holds it;
// 1: load st.next by TMA (a bxc x byc box, x rounded down to the TMA alignment);
// 3: copy st.next cooperatively (pitch = its width); 2: too large for shared
// memory, samples read the global plane.
template <typename C, int NP, typename SC>
__device__ void plan_window(PointState<C, NP, SC>& st, int xc, int yc, int r, int W, int H,
                            const WaveTiles& t, int xalign) {
  int x0, x1, y0, y1;
  st.inside = 0;
  if (!needed_range<C, NP>(st.p, xc, yc, r, W, H, &x0, &x1, &y0, &y1, &st.inside)) {
    st.stage = 2;
    return;
  }
  const Window& cw = st.win;
  if (cw.w > 0 && x0 >= cw.x0 && y0 >= cw.y0 && x1 < cw.x0 + cw.w && y1 < cw.y0 + cw.h) {
    st.stage = 0;
    return;
  }
  const int nw = x1 - x0 + 1, nh = y1 - y0 + 1;
  if (t.coef_tma && nw + xalign - 1 <= t.bxc && nh <= t.byc) {
    // centre the needed range in the box so the next iterations reuse it
    int bx = x0 - (t.bxc - nw - (xalign - 1)) / 2;
    bx -= ((bx % xalign) + xalign) % xalign;
    if (bx + t.bxc - 1 < x1) bx += xalign;
    const int by = y0 - (t.byc - nh) / 2;
    st.next = Window{bx, by, t.bxc, t.byc};
    st.stage = 1;
    return;
  }
  if (static_cast<int64_t>(nw) * nh <= static_cast<int64_t>(t.bxc) * t.byc) {
    st.next = Window{x0, y0, nw, nh};
    st.stage = 3;
    return;
  }
  st.stage = 2;
}

// Warp 0 after the reference reduction: mean and contrast of f, the Hessian and
// its inverse. out: [H moments (3 NMOM), sum SD f', sum SD, sum f', sum f'^2].
// FP64 path: the Hessian in FP64 and its inverse by invert_spd_warp. Mixed path:
// the Jacobi-scaled FP32 inverse; a scaled pivot below 1e-5 (H too
// ill-conditioned for FP32) switches to the same scaled inverse in FP64. Sets
// st.ctl: 0 ok, 3 flat, 4 singular (a pivot <= 1e-12 of the largest diagonal
// entry of H).
template <typename C, int NP, int NMOM, int M2, bool ANYCOST, typename SC>
__device__ void finish_reference(PointState<C, NP, SC>& st, const C* out, int N, int lane, int cost) {
  const C sf = out[3 * NMOM + 2 * NP];
  const C sff = out[3 * NMOM + 2 * NP + 1];
  const C mu = sf / static_cast<C>(N);
  const C df = sqrt(fmax(sff - sf * mu, C(0)));
  if (is_flat<C>(df, mu + st.f0, N)) {
    if (lane == 0) st.ctl = 3;
    return;
  }
  auto hget = [&](int ca, int cb) -> C {
    return out[(sd_t(ca) + sd_t(cb)) * NMOM + mono(sd_i(ca) + sd_i(cb), sd_j(ca) + sd_j(cb), M2)];
  };
  double ratio;
  if constexpr (std::is_same<SC, Refined64>::value) {
    for (int e = lane; e < NP * NP; e += 32) st.sv.H[e] = static_cast<double>(hget(e / NP, e % NP));
    float rf;
    if (invert_scaled_warp<float, NP>(hget, st.sv.X, lane, &rf) < 1e-5f)
      invert_scaled_fp64<NP, NMOM, M2>(out, st.sv.X, lane, &rf);
    ratio = rf;
  } else if constexpr (sizeof(SC) == sizeof(double)) {
    for (int e = lane; e < NP * NP; e += 32) st.sv.H[e] = static_cast<double>(hget(e / NP, e % NP));
    __syncwarp();
    ratio = invert_spd_warp<SC, NP>(st.sv.H, st.sv.X, lane);
  } else {
    float rf;
    if (invert_scaled_warp<float, NP>(hget, st.sv.X, lane, &rf) < 1e-5f)
      invert_scaled_fp64<NP, NMOM, M2>(out, st.sv.X, lane, &rf);
    ratio = rf;
  }
  if (lane < NP) {
    st.sds[lane] = out[3 * NMOM + NP + lane];
    // ZNSSD: sum SD (f' - mu) = sum SD fbar; NSSD and SSD: sum SD f'
    st.sdf[lane] = out[3 * NMOM + lane] - ((!ANYCOST || cost == DIC_COST_ZNSSD) ? mu : C(0)) * out[3 * NMOM + NP + lane];
  }
  if (lane == 0) {
    st.mu = mu;
    st.delta_f = df;
    if constexpr (std::is_same<SC, Refined64>::value) {
      const double mu64 = static_cast<double>(sf) / static_cast<double>(N);
      st.mu64 = mu64;
      st.delta_f64 = sqrt(fmax(static_cast<double>(sff) - static_cast<double>(sf) * mu64, 0.0));
    }
    if (ANYCOST) {
      st.sf = sf;
      st.sff = sff;
    }
    st.ctl = ratio > 1e-12 ? 0 : 4;
  }
  __syncwarp();
}

// Warp 0 after an iteration's reduction. out: [sum g', sum g'^2, sum SD g', bad].
// b = sum SD e, one component per lane (f' = f - f0, g' = g - f0 with f0 the
// reference gray level at the centre, so that the large common level cancels):
//   ZNSSD  b = sum SD (f - f_m) - (df/dg) sum SD (g - g_m),
//   NSSD   b = sum SD f' - r sum SD g' + f0 (1 - r) sum SD, r = ||f|| / ||g||,
//   SSD    b = sum SD f' - sum SD g'.
// FP64 path: dp0 = -X b in FP64, then one refinement step dp = dp0 - X (b + H dp0).
// Mixed path: dp = -H^-1 b in FP32, b shared by shuffles (the precision of the
// solve sets the rate of convergence, not the root, which b alone fixes). Lane 0
// composes p <- p o dp^-1. Returns (on every lane) 0 continue, 1 converged,
// 2 flat, 5 out of bounds.
template <typename C, int NP, bool ANYCOST, typename SC>
__device__ int gauss_newton_update(PointState<C, NP, SC>& st, const C* out, int N, C r, C thr2, int lane,
                                   int cost) {
  if (out[2 + NP] > C(0.5)) return 5;
  const C nu = out[0] * (C(1) / static_cast<C>(N));  // mean of g' = g - f0
  const C dg2 = fmax(out[1] - out[0] * nu, C(0));
  // flat: dg / sqrt(N) <= 1e-6 max(|mean|, 1), compared squared
  const C gm = fmax(fabs(nu + st.f0), C(1));
  if (dg2 <= C(1e-12) * static_cast<C>(N) * gm * gm) return 2;
  const C ratio = st.delta_f * rsqrt(dg2);
  // coefficients of b = sdf - kg sum SD g' + kc sum SD
  C kg = ratio, kc = ratio * nu;
  if (!ANYCOST) {
  } else if (cost == DIC_COST_SSD) {
    kg = C(1);
    kc = C(0);
  } else if (cost == DIC_COST_NSSD) {
    const C f0 = st.f0, n = static_cast<C>(N);
    const C nf2 = st.sff + C(2) * f0 * st.sf + n * f0 * f0;   // ||f||^2
    const C ng2 = out[1] + C(2) * f0 * out[0] + n * f0 * f0;  // ||g||^2
    const C nf = sqrt(nf2), ng = sqrt(ng2);
    kg = nf / ng;
    // 1 - r from the difference of the squared norms (the N f0^2 terms cancel)
    kc = f0 * ((out[1] - st.sff) + C(2) * f0 * (out[0] - st.sf)) / (ng * (ng + nf));
  }
  C d;
  if constexpr (std::is_same<SC, Refined64>::value) {
    // H dp = -b by one step of iterative refinement: x0 = -X b with the FP32 inverse,
    // the residual r = b + H x0 in FP64 against the FP64 Hessian, x = x0 - X r; the
    // error of x is about the square of x0's relative error (a few FP32 roundings times
    // the scaled condition number), far below FP32 rounding
    const C bcf = lane < NP ? st.sdf[lane] - ratio * (out[2 + lane] - nu * st.sds[lane]) : C(0);
    const int row = lane < NP ? lane : 0;
    C x0 = C(0);
#pragma unroll
    for (int m = 0; m < NP; ++m) x0 -= st.sv.X[m * NP + row] * __shfl_sync(0xffffffffu, bcf, m);
    double res = static_cast<double>(bcf);
#pragma unroll
    for (int m = 0; m < NP; ++m)
      res += st.sv.H[row * NP + m] * static_cast<double>(__shfl_sync(0xffffffffu, x0, m));
    const C rf = static_cast<C>(res);
    C dx = C(0);
#pragma unroll
    for (int m = 0; m < NP; ++m) dx -= st.sv.X[m * NP + row] * __shfl_sync(0xffffffffu, rf, m);
    d = lane < NP ? static_cast<C>(static_cast<double>(x0) + static_cast<double>(dx)) : C(0);
  } else if constexpr (sizeof(SC) == sizeof(double)) {
    double bc = 0.0;
    if (lane < NP)
      bc = static_cast<double>(ANYCOST ? st.sdf[lane] - kg * out[2 + lane] + kc * st.sds[lane]
                                       : st.sdf[lane] - ratio * (out[2 + lane] - nu * st.sds[lane]));
    if (lane < NP) st.sv.bvec[lane] = bc;
    __syncwarp();
    double d0 = 0.0;
    if (lane < NP) {
#pragma unroll
      for (int m = 0; m < NP; ++m) d0 -= st.sv.X[lane * NP + m] * st.sv.bvec[m];
      st.sv.dvec[lane] = d0;
    }
    __syncwarp();
    double res = bc;
    if (lane < NP) {
#pragma unroll
      for (int m = 0; m < NP; ++m) res += st.sv.H[lane * NP + m] * st.sv.dvec[m];
    }
    __syncwarp();
    if (lane < NP) st.sv.bvec[lane] = res;
    __syncwarp();
    double dpc = d0;
    if (lane < NP) {
#pragma unroll
      for (int m = 0; m < NP; ++m) dpc -= st.sv.X[lane * NP + m] * st.sv.bvec[m];
    }
    d = static_cast<C>(dpc);
  } else {
    const C bc = lane >= NP ? C(0)
                 : ANYCOST ? st.sdf[lane] - kg * out[2 + lane] + kc * st.sds[lane]
                           : st.sdf[lane] - ratio * (out[2 + lane] - nu * st.sds[lane]);
    const int row = lane < NP ? lane : 0;
    C acc = C(0);
#pragma unroll
    for (int m = 0; m < NP; ++m) acc -= st.sv.X[m * NP + row] * __shfl_sync(0xffffffffu, bc, m);
    d = lane < NP ? acc : C(0);
  }
  if (lane < NP) st.dp[lane] = d;
  // ||dp||^2 with weights 1, r^2, r^4 on the rigid, affine and quadratic terms
  const C wgt = lane < 2 ? C(1) : (lane < 6 ? r * r : r * r * r * r);
  C n2 = lane < NP ? wgt * d * d : C(0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
  __syncwarp();
  if (lane == 0) compose_inverse<C, NP>(st.p, st.dp);
  __syncwarp();
  return n2 < thr2 ? 1 : 0;
}

// Levenberg-Marquardt state of a point (Sec. 2.2): the undamped Hessian and its
// inverse (the layout of the solve state's inverse), the best trial so far (its warp,
// right-hand side, cost and squared undamped step) and the damping; empty for
// Gauss-Newton.
constexpr float kLmLambda0 = 1e-3f, kLmFactor = 10.0f;
template <typename C, int NP, bool LM>
struct LmState {};
template <typename C, int NP>
struct LmState<C, NP, true> {
  C H[NP * NP];
  C X0[NP * NP];
  C b_best[NP];
  C p_best[kMaxParams];
  C lam, c_best, s2_best;
  int has_best;
};

// -X0 b (the undamped step) on lanes < NP; X0 column-major on the mixed path (shared
// through b by shuffles), row-major on the FP64 path
template <typename C, int NP>
__device__ __forceinline__ C undamped_step(const C* X0, C b, int lane) {
  const int row = lane < NP ? lane : 0;
  C acc = C(0);
#pragma unroll
  for (int m = 0; m < NP; ++m) {
    const C bm = __shfl_sync(0xffffffffu, b, m);
    acc -= (sizeof(C) == sizeof(double) ? X0[row * NP + m] : X0[m * NP + row]) * bm;
  }
  return lane < NP ? acc : C(0);
}

// squared ||d||_s of reading R7 over the warp (every lane gets it)
template <typename C>
__device__ __forceinline__ C step_norm2(C d, C r, int lane, int NP) {
  const C wgt = lane < 2 ? C(1) : (lane < 6 ? r * r : r * r * r * r);
  C n2 = lane < NP ? wgt * d * d : C(0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
  return n2;
}

// The out-of-line FP64 inverse of a scaled matrix read through hget (the FP32 one
// met a tiny pivot).
template <int N, typename HGet>
__device__ __noinline__ void invert_scaled_fp64_from(HGet hget, float* X, int lane, float* ratio) {
  invert_scaled_warp<double, N>(hget, X, lane, ratio);
}

// Warp 0 after an iteration's reduction, Levenberg-Marquardt: out = [sum g', sum g'^2,
// sum SD g', bad, sum f' g']. At the trial: the cost (Eq. 2-4, from the sums) and the
// undamped Gauss-Newton step -H^-1 b. The trial is kept when it is the first, lowers
// the cost or shortens that step (the inverse-compositional root and the minimum of
// the cost differ at second order); keeping divides lambda by 10, refusing multiplies
// it by 10. Converged when the best trial's undamped step is below the threshold:
// that step is applied. Otherwise the damped step solves (H + lambda diag H) dp =
// -b_best (its inverse formed again). The next trial is p_best o dp^-1. Returns like
// gauss_newton_update.
template <typename C, int NP>
__device__ int lm_update(PointState<C, NP>& st, LmState<C, NP, true>& lm, const C* out, int N, C r, C thr2,
                         int lane, int cost) {
  if (out[2 + NP] > C(0.5)) return 5;
  const C n = static_cast<C>(N);
  const C nu = out[0] * (C(1) / n);
  const C dg2 = fmax(out[1] - out[0] * nu, C(0));
  const C gm = fmax(fabs(nu + st.f0), C(1));
  if (dg2 <= C(1e-12) * n * gm * gm) return 2;
  const C sfg = out[3 + NP];
  const C f0 = st.f0;
  C kg, kc, cval;
  if (cost == DIC_COST_SSD) {
    kg = C(1);
    kc = C(0);
    cval = st.sff - C(2) * sfg + out[1];                        // sum (f' - g')^2
  } else if (cost == DIC_COST_NSSD) {
    const C nf2 = st.sff + C(2) * f0 * st.sf + n * f0 * f0;
    const C ng2 = out[1] + C(2) * f0 * out[0] + n * f0 * f0;
    const C nf = sqrt(nf2), ng = sqrt(ng2);
    kg = nf / ng;
    kc = f0 * ((out[1] - st.sff) + C(2) * f0 * (out[0] - st.sf)) / (ng * (ng + nf));
    const C sfgf = sfg + f0 * (out[0] + st.sf) + n * f0 * f0;    // sum f g
    cval = C(2) - C(2) * sfgf / (nf * ng);
  } else {
    const C dg = sqrt(dg2);
    kg = st.delta_f / dg;
    kc = kg * nu;
    cval = C(2) - C(2) * (sfg - st.mu * out[0]) / (st.delta_f * dg);   // sum fbar gbar = sum f'g' - mu sum g'
  }
  const C bk = lane < NP ? st.sdf[lane] - kg * out[2 + lane] + kc * st.sds[lane] : C(0);
  const C s2 = step_norm2<C>(undamped_step<C, NP>(lm.X0, bk, lane), r, lane, NP);
  const bool keep = !lm.has_best || cval < lm.c_best || s2 < lm.s2_best;   // the same on every lane
  if (keep) {
    if (lane < NP) lm.b_best[lane] = bk;
    if (lane < kMaxParams) lm.p_best[lane] = st.p[lane];
  }
  __syncwarp();
  if (lane == 0) {
    if (keep) {
      lm.c_best = cval;
      lm.s2_best = s2;
      lm.has_best = 1;
      lm.lam = lm.lam / C(kLmFactor);
    } else {
      lm.lam = lm.lam * C(kLmFactor);
    }
  }
  __syncwarp();
  const bool converged = lm.s2_best < thr2;
  const C bb = lane < NP ? lm.b_best[lane] : C(0);
  C d;
  if (converged) {
    d = undamped_step<C, NP>(lm.X0, bb, lane);
  } else {
    const C lam = lm.lam;
    if constexpr (sizeof(C) == sizeof(double)) {
      for (int e = lane; e < NP * NP; e += 32)
        st.sv.H[e] = lm.H[e] * ((e / NP == e % NP) ? C(1) + lam : C(1));
      __syncwarp();
      invert_spd_warp<C, NP>(st.sv.H, st.sv.X, lane);
    } else {
      auto hget = [&](int i, int j) -> float { return lm.H[i * NP + j] * (i == j ? 1.0f + lam : 1.0f); };
      float rf;
      if (invert_scaled_warp<float, NP>(hget, st.sv.X, lane, &rf) < 1e-5f)
        invert_scaled_fp64_from<NP>(hget, st.sv.X, lane, &rf);
    }
    __syncwarp();
    d = undamped_step<C, NP>(st.sv.X, bb, lane);   // the same product with the damped inverse
  }
  if (lane < NP) st.dp[lane] = d;
  __syncwarp();
  if (lane == 0) {
    for (int c = 0; c < NP; ++c) st.p[c] = lm.p_best[c];
    compose_inverse<C, NP>(st.p, st.dp);
  }
  __syncwarp();
  return converged ? 1 : 0;
}

// Two values that go through the same arithmetic (an x quantity with its y
// counterpart): on the mixed path one packed FP32x2 instruction per operation,
// rounded exactly like the two scalar operations; on the FP64 path two scalar ones.
template <typename T>
struct alignas(2 * sizeof(T)) Pair {
  T x, y;
};
template <typename T>
__device__ __forceinline__ Pair<T> pair(T a, T b) {
  return Pair<T>{a, b};
}
template <typename T>
__device__ __forceinline__ Pair<T> pfma(Pair<T> a, Pair<T> b, Pair<T> c) {   // a b + c
  return Pair<T>{fma(a.x, b.x, c.x), fma(a.y, b.y, c.y)};
}
template <typename T>
__device__ __forceinline__ Pair<T> pmul(Pair<T> a, Pair<T> b) {
  return Pair<T>{a.x * b.x, a.y * b.y};
}
template <typename T>
__device__ __forceinline__ Pair<T> padd(Pair<T> a, Pair<T> b) {
  return Pair<T>{a.x + b.x, a.y + b.y};
}
template <typename T>
__device__ __forceinline__ Pair<T> psub(Pair<T> a, Pair<T> b) {
  return Pair<T>{a.x - b.x, a.y - b.y};
}
__device__ __forceinline__ unsigned long long pair_bits(Pair<float> a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ Pair<float> bits_pair(unsigned long long r) {
  Pair<float> a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
template <>
__device__ __forceinline__ Pair<float> pfma<float>(Pair<float> a, Pair<float> b, Pair<float> c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pair_bits(a)), "l"(pair_bits(b)), "l"(pair_bits(c)));
  return bits_pair(d);
}
template <>
__device__ __forceinline__ Pair<float> pmul<float>(Pair<float> a, Pair<float> b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pair_bits(a)), "l"(pair_bits(b)));
  return bits_pair(d);
}
template <>
__device__ __forceinline__ Pair<float> padd<float>(Pair<float> a, Pair<float> b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pair_bits(a)), "l"(pair_bits(b)));
  return bits_pair(d);
}
template <>
__device__ __forceinline__ Pair<float> psub<float>(Pair<float> a, Pair<float> b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pair_bits(a)), "l"(pair_bits(b)));
  return bits_pair(d);
}

// floor of both values and their integer parts. FP32 (|x| < 2^22): x + 1.5 * 2^23
// rounded toward minus infinity is floor(x) + 1.5 * 2^23 exactly, an integer whose
// low mantissa bits hold floor(x); one packed add, one packed subtract and two
// integer subtracts replace two roundings and two conversions. FP64: floor().
template <typename T>
__device__ __forceinline__ Pair<T> pfloor(Pair<T> x, int& ix, int& iy) {
  const T fx = floor(x.x), fy = floor(x.y);
  ix = static_cast<int>(fx);
  iy = static_cast<int>(fy);
  return Pair<T>{fx, fy};
}
template <>
__device__ __forceinline__ Pair<float> pfloor<float>(Pair<float> x, int& ix, int& iy) {
  constexpr float kMagic = 12582912.0f;   // 1.5 * 2^23
  unsigned long long d;
  asm("add.rm.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pair_bits(x)), "l"(pair_bits(Pair<float>{kMagic, kMagic})));
  const Pair<float> t = bits_pair(d);
  ix = __float_as_int(t.x) - 0x4B400000;
  iy = __float_as_int(t.y) - 0x4B400000;
  return psub(t, Pair<float>{kMagic, kMagic});
}

// bspline_weights6 of two offsets at once (x in .x, y in .y), the same arithmetic
template <typename T>
__device__ __forceinline__ void bspline_weights6_pair(Pair<T> t, Pair<T>& w0, Pair<T>& w1, Pair<T>& w2,
                                                      Pair<T>& w3) {
  const Pair<T> s = psub(pair(T(1), T(1)), t);
  const Pair<T> t2 = pmul(t, t), s2 = pmul(s, s);
  w3 = pmul(t2, t);
  w0 = pmul(s2, s);
  w1 = pfma(t2, pfma(pair(T(3), T(3)), t, pair(T(-6), T(-6))), pair(T(4), T(4)));
  w2 = pfma(s2, pfma(pair(T(3), T(3)), s, pair(T(-6), T(-6))), pair(T(4), T(4)));
}

// Keys' cubic convolution weights (a = -1/2) of two offsets, times 2, in the layout
// of bspline_weights6_pair: w0..w3 weigh the samples at -1, 0, 1, 2, so that the
// interpolated value is the weighted sum over the 4 x 4 support divided by 4.
//   2 K(1 + t) = -t s^2,  2 K(t) = t^2 (3t - 5) + 2,  2 K(s) = s^2 (3s - 5) + 2,
//   2 K(1 + s) = -s t^2,  s = 1 - t
template <typename T>
__device__ __forceinline__ void keys_weights2_pair(Pair<T> t, Pair<T>& w0, Pair<T>& w1, Pair<T>& w2,
                                                   Pair<T>& w3) {
  const Pair<T> s = psub(pair(T(1), T(1)), t);
  const Pair<T> t2 = pmul(t, t), s2 = pmul(s, s);
  const Pair<T> m1 = pair(T(-1), T(-1));
  w0 = pmul(pmul(s2, t), m1);
  w3 = pmul(pmul(t2, s), m1);
  w1 = pfma(t2, pfma(pair(T(3), T(3)), t, pair(T(-5), T(-5))), pair(T(2), T(2)));
  w2 = pfma(s2, pfma(pair(T(3), T(3)), s, pair(T(-5), T(-5))), pair(T(2), T(2)));
}
template <typename T>
__device__ __forceinline__ void keys_weights2(T t, T& w0, T& w1, T& w2, T& w3) {
  const T s = T(1) - t;
  const T t2 = t * t, s2 = s * s;
  w0 = -(s2 * t);
  w3 = -(t2 * s);
  w1 = t2 * (T(3) * t - T(5)) + T(2);
  w2 = s2 * (T(3) * s - T(5)) + T(2);
}

// Sums over one thread's column of subset pixels at the warp given by
// (ax, bx, cxq; ay, by, cyq): x = ax + dy (bx + cxq dy), y = ay + dy (by + cyq dy)
// relative to the centre. The support of a sample at (ix + tx, iy + ty) starts at
// base + iy * ld + ix (row iy - 1, column ix - 1 of the plane). Consecutive rows of
// a column usually step one coefficient row down with the same ix, so the four
// rows of the support stay in registers (rotated by the 4-way unrolled loop) and
// only the new row is loaded; anything else reloads all four.
// fin = false: acc = [sum g', sum g'^2, sum fx g' dy^j (j <= D), sum fy g' dy^j]
//              (FG: then sum f' g', which the Levenberg-Marquardt cost needs)
// fin = true:  acc = [sum g', sum g'^2, sum f' g'] (the final pass; one copy of the
// unrolled loop serves both, fin being the same for the whole block)
// GEN: the interpolant is a runtime choice (keys: bicubic convolution on gray
// levels; otherwise the B-spline), else the B-spline is compiled in.
template <typename T, int D, bool FG, bool GEN>
__device__ __forceinline__ void sample_column(const T* __restrict__ base, int ld, T ax, T bx, T cxq,
                                              T ay, T by, T cyq, T xlo, T xhi, T ylo, T yhi, T f0,
                                              int row0, int row1, int r, int S, int col,
                                              const T* s_f, const Pair<T>* s_fg, bool fin, bool inside,
                                              bool keys, T* acc, T& bad) {
  T c0[4], c1[4], c2[4], c3[4];
  Pair<T> sd[D + 1];   // sum fx g' dy^j in .x, sum fy g' dy^j in .y
#pragma unroll
  for (int j = 0; j <= D; ++j) sd[j] = pair(T(0), T(0));
  const Pair<T> a2 = pair(ax, ay), b2 = pair(bx, by), cq2 = pair(cxq, cyq);
  int pix_ix = -0x40000000, pix_iy = -0x40000000;
  T dyr = static_cast<T>(row0 - r);                  // dy of the next row, counted in T (exact)
  const Pair<T>* fgp = s_fg + row0 * S + col;       // gradients of the next row's pixel
  const T* fpp = s_f + row0 * S + col;            // its reference gray level f - f0
  auto step = [&](T (&A)[4], T (&B)[4], T (&Cc)[4], T (&Dn)[4]) {
    const T dyv = dyr;
    dyr += T(1);
    const Pair<T> fg = *fgp;
    fgp += S;
    const T fr = *fpp;
    fpp += S;
    const Pair<T> dy2 = pair(dyv, dyv);
    const Pair<T> xy = D >= 2 ? pfma(dy2, pfma(cq2, dy2, b2), a2) : pfma(dy2, b2, a2);
    const T xl = xy.x, yl = xy.y;
    if (!inside && !(xl >= xlo && xl < xhi && yl >= ylo && yl < yhi)) {
      bad += T(1);
      pix_ix = -0x40000000;
      return;
    }
    int ix, iy;
    const Pair<T> fl = pfloor<T>(xy, ix, iy);
    const T* b = base + (iy * ld + ix);
    if (!(ix == pix_ix && iy == pix_iy + 1)) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        A[k] = b[k];
        B[k] = b[ld + k];
        Cc[k] = b[2 * ld + k];
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) Dn[k] = b[3 * ld + k];
    pix_ix = ix;
    pix_iy = iy;
    Pair<T> w0, w1, w2, w3;
    if (GEN && keys)
      keys_weights2_pair<T>(psub(xy, fl), w0, w1, w2, w3);
    else
      bspline_weights6_pair<T>(psub(xy, fl), w0, w1, w2, w3);
    const T wx0 = w0.x, wx1 = w1.x, wx2 = w2.x, wx3 = w3.x;
    const T wy0 = w0.y, wy1 = w1.y, wy2 = w2.y, wy3 = w3.y;
    const T r0 = wx0 * A[0] + wx1 * A[1] + wx2 * A[2] + wx3 * A[3];
    const T r1 = wx0 * B[0] + wx1 * B[1] + wx2 * B[2] + wx3 * B[3];
    const T r2 = wx0 * Cc[0] + wx1 * Cc[1] + wx2 * Cc[2] + wx3 * Cc[3];
    const T r3 = wx0 * Dn[0] + wx1 * Dn[1] + wx2 * Dn[2] + wx3 * Dn[3];
    const T gp = (wy0 * r0 + wy1 * r1 + wy2 * r2 + wy3 * r3) * (GEN && keys ? T(0.25) : T(1) / T(36)) - f0;
    acc[0] += gp;
    acc[1] += gp * gp;
    if (fin) {
      acc[2] += gp * fr;
    } else {
      const Pair<T> g2 = pmul(pair(gp, gp), fg);   // (fx g', fy g')
      if (FG) acc[2 + 2 * (D + 1)] += gp * fr;
      sd[0] = padd(sd[0], g2);
      Pair<T> dyp = dy2;
#pragma unroll
      for (int j = 1; j <= D; ++j) {
        sd[j] = pfma(g2, dyp, sd[j]);
        if (j < D) dyp = pmul(dyp, dy2);
      }
    }
  };
  for (int row = row0; row < row1; row += 4) {
    step(c0, c1, c2, c3);
    if (row + 1 < row1) step(c1, c2, c3, c0);
    if (row + 2 < row1) step(c2, c3, c0, c1);
    if (row + 3 < row1) step(c3, c0, c1, c2);
  }
  if (!fin) {
#pragma unroll
    for (int j = 0; j <= D; ++j) {
      acc[2 + j] += sd[j].x;
      acc[2 + D + 1 + j] += sd[j].y;
    }
  }
}

// The rare path (window too large for shared memory): every sample reads its
// 4 x 4 support from the global plane; a plain loop, light on registers, kept out
// of line so that it does not sit in the instruction stream of the common path.
template <typename T, int D, bool FG>
__device__ __noinline__ void sample_column_global(const T* __restrict__ base, int64_t ld, T ax,
                                                     T bx, T cxq, T ay, T by, T cyq, T xlo, T xhi,
                                                     T ylo, T yhi, T f0, int row0, int row1, int r,
                                                     int S, int col, const T* s_f, const Pair<T>* s_fg,
                                                     bool fin, bool keys, T* acc, T& bad) {
  for (int row = row0; row < row1; ++row) {
    const T dyv = static_cast<T>(row - r);
    const T xl = ax + dyv * (bx + cxq * dyv);
    const T yl = ay + dyv * (by + cyq * dyv);
    if (!(xl >= xlo && xl < xhi && yl >= ylo && yl < yhi)) {
      bad += T(1);
      continue;
    }
    const T xf = floor(xl), yf = floor(yl);
    const T* b = base + (static_cast<int64_t>(yf) * ld + static_cast<int64_t>(xf));
    T wx0, wx1, wx2, wx3, wy0, wy1, wy2, wy3;
    if (keys) {
      keys_weights2<T>(xl - xf, wx0, wx1, wx2, wx3);
      keys_weights2<T>(yl - yf, wy0, wy1, wy2, wy3);
    } else {
      bspline_weights6<T>(xl - xf, wx0, wx1, wx2, wx3);
      bspline_weights6<T>(yl - yf, wy0, wy1, wy2, wy3);
    }
    T g = T(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const T* rj = b + j * ld;
      const T wy = j == 0 ? wy0 : j == 1 ? wy1 : j == 2 ? wy2 : wy3;
      g += wy * (wx0 * rj[0] + wx1 * rj[1] + wx2 * rj[2] + wx3 * rj[3]);
    }
    const T gp = g * (keys ? T(0.25) : T(1) / T(36)) - f0;
    acc[0] += gp;
    acc[1] += gp * gp;
    if (fin) {
      acc[2] += gp * s_f[row * S + col];
    } else {
      const Pair<T> fg = s_fg[row * S + col];
      const T gxv = gp * fg.x, gyv = gp * fg.y;
      if (FG) acc[2 + 2 * (D + 1)] += gp * s_f[row * S + col];
      T dyp = T(1);
#pragma unroll
      for (int j = 0; j <= D; ++j) {
        acc[2 + j] += gxv * dyp;
        acc[2 + D + 1 + j] += gyv * dyp;
        dyp *= dyv;
      }
    }
  }
}

// resident blocks per SM the register budget is sized for
template <typename T, int NT>
struct WaveOccupancy;
template <>
struct WaveOccupancy<float, 128> { static constexpr int kBlocks = 7; };   // 72 registers (12 parameters: 6, below)
template <>
struct WaveOccupancy<float, 64> { static constexpr int kBlocks = 14; };
template <>
struct WaveOccupancy<double, 128> { static constexpr int kBlocks = 4; };
template <>
struct WaveOccupancy<double, 64> { static constexpr int kBlocks = 8; };

// MODE 0: Gauss-Newton, ZNSSD only (the default, leanest); 1: Gauss-Newton, any cost;
// 2: Levenberg-Marquardt, any cost
// Resident blocks the registers are sized for. The quadratic FP32 kernels take fewer
// blocks than the others, for registers that spare them spills: 6 of 128 threads (at
// 7 its register cap costs more in spills than the extra block gains) and 10 of 64
// (96 registers; at 14 they spill about 100 bytes a thread)
template <typename T, int NP, int NT>
constexpr int wave_min_blocks() {
  if (sizeof(T) == 4 && NP == 12) return NT == 128 ? 6 : 10;
  return WaveOccupancy<T, NT>::kBlocks;
}

template <typename T, int NP, int NT, int MODE>
__global__ void __launch_bounds__(NT, wave_min_blocks<T, NP, NT>())
    wave_kernel(WaveArgs<T> a, const __grid_constant__ CUtensorMap tm_cref,
                const __grid_constant__ CUtensorMap tm_cdef, const __grid_constant__ CUtensorMap tm_gray) {
  using C = T;  // working precision of the per-point control arithmetic
  constexpr bool LM = MODE == 2;
  constexpr bool ANYCOST = MODE == 1 || MODE == 2;
  constexpr bool GEN = MODE == 1 || MODE == 2;       // the interpolant is a runtime choice
  constexpr bool S64 = MODE == 3;                    // mixed path with FP64 solves and ZNCC
  using SC = typename std::conditional<S64, Refined64, C>::type;
  const bool keys = GEN && a.interp == DIC_BICUBIC;
  constexpr int D = Shape<NP>::D;
  constexpr int M2 = 2 * D;
  constexpr int NMOM = (M2 + 1) * (M2 + 2) / 2;
  constexpr int NV_PRE = 3 * NMOM + 2 * NP + 2;  // H moments, sum SD f', sum SD, sum f', sum f'^2
  constexpr int NV_IT = 4 + NP;                  // sum g', sum g'^2, sum SD g', bad samples, sum f'g'
  constexpr int NV_FIN = 4;                      // sum g', sum g'^2, sum f' g', bad samples
  constexpr int NACC = 2 + 2 * (D + 1) + 1;
  constexpr int XALIGN = 16 / static_cast<int>(sizeof(T));   // TMA x alignment of the coefficient planes
  constexpr int NW = NT / 32;                                 // warps per block

  extern __shared__ __align__(128) unsigned char smem_raw[];
  const WaveTiles& tl = a.tiles;
  const int S = a.S, r = a.r, N = S * S;
  // reference gradients (fx, fy) of the subset pixels, interleaved
  Pair<T>* s_fg = reinterpret_cast<Pair<T>*>(smem_raw + tl.off_fg);
  T* s_f = reinterpret_cast<T*>(smem_raw + tl.off_f);   // f - f0 of the subset pixels
  T* s_win = reinterpret_cast<T*>(smem_raw + tl.off_win);
  unsigned char* s_gray = smem_raw + tl.off_gray;
  const int gdt = a.ref_gray.dtype;
  const int gpitch = tl.bxg * tl.gray_es;

  __shared__ T s_part[NW][NV_PRE];
  __shared__ C s_out[NV_PRE];
  __shared__ PointState<C, NP, SC> st;
  __shared__ LmState<C, NP, LM> lms;
  __shared__ __align__(8) uint64_t s_bar;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cur = a.k % 3, nxt = (a.k + 1) % 3, old = (a.k + 2) % 3;
  if (blockIdx.x == 0 && tid == 0) {
    a.counters[kCount + old] = 0;
    a.counters[kWork + nxt] = 0;
    a.wave_sizes[a.k] = a.counters[kCount + cur];
  }
  const int n_front = a.counters[kCount + cur];
  if (tid == 0) mbar_init(&s_bar, 1);
  __syncthreads();
  uint32_t bar_phase = 0;
  // every thread waits for the pending TMA transaction; a lost wait ends the block
  // (a.expire_waits: the wait gives up without polling; the drain below still lets
  // the copy land before the block exits)
  auto tma_wait = [&]() -> bool {
    const bool ok = !a.expire_waits && mbar_wait_bounded(&s_bar, bar_phase);
    bar_phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(&a.counters[kError], 1);
        mbar_wait_bounded(&s_bar, bar_phase ^ 1u);   // let a late copy land before leaving
      }
      return false;
    }
    return true;
  };

  const int col = tid % S;
  const int band = tid / S;
  const int row0 = band < a.bands ? band * a.band_h : S;
  const int row1 = min(row0 + a.band_h, S);
  const T dxv = static_cast<T>(col - r);
  T dxp[M2 + 1];
  dxp[0] = T(1);
#pragma unroll
  for (int i = 1; i <= M2; ++i) dxp[i] = dxp[i - 1] * dxv;

  // warp partials of entries [base, base + count) of a reduction vector from the
  // values v[0..K) of every thread (entries count..K-1 are padding)
  auto parts = [&](auto& v, int base, int count) {
    constexpr int K = sizeof(v) / sizeof(v[0]);
    constexpr int SH = 5 - Log2<K>::kValue;
    const T sum = warp_transpose_sum<T, K>(v, lane);
    const int e = lane >> SH;
    if ((lane & ((1 << SH) - 1)) == 0 && e < count) s_part[warp][base + e] = sum;
  };
  // warp 0: cross-warp sums into s_out[0..nv)
  auto gather = [&](int nv) {
    for (int i = lane; i < nv; i += 32) {
      C sacc = C(0);
#pragma unroll
      for (int w = 0; w < NW; ++w) sacc += s_part[w][i];
      s_out[i] = sacc;
    }
    __syncwarp();
  };

  for (;;) {
    // ---- 1. next point and its starting warp (warp 0)
    if (warp == 0) {
      int item = 0;
      if (lane == 0) item = atomicAdd(&a.counters[kWork + cur], 1);
      item = __shfl_sync(0xffffffffu, item, 0);
      if (item < n_front) {
        const int q = a.cur[item];
        const int gi = q % a.nx, gj = q / a.nx;
        int best = -1;
        if (a.k == 0) {
          best = q;
        } else {
          // the accepted neighbour from an earlier wave with the highest ZNCC
          // (ties to the lower index); lanes 0-3 look at left, right, up, down
          int nb = -1;
          if (lane == 0 && gi > 0) nb = q - 1;
          if (lane == 1 && gi < a.nx - 1) nb = q + 1;
          if (lane == 2 && gj > 0) nb = q - a.nx;
          if (lane == 3 && gj < a.ny - 1) nb = q + a.nx;
          float z = -3.0f;
          int cand = 0x7fffffff;
          if (nb >= 0) {
            const int64_t rec = a.pts.accept[nb];
            if (rec >= 0 && static_cast<int>(rec >> 32) < a.k) {
              z = __int_as_float(static_cast<int>(rec & 0xffffffffLL));
              cand = nb;
            }
          }
#pragma unroll
          for (int o = 1; o <= 2; o <<= 1) {
            const float oz = __shfl_xor_sync(0xffffffffu, z, o);
            const int oc = __shfl_xor_sync(0xffffffffu, cand, o);
            if (oz > z || (oz == z && oc < cand)) {
              z = oz;
              cand = oc;
            }
          }
          best = __shfl_sync(0xffffffffu, cand, 0);
          if (best == 0x7fffffff) best = -1;
        }
        if (lane < NP)
          st.dp[lane] = best >= 0 ? static_cast<C>(a.pts.p[static_cast<int64_t>(best) * NP + lane]) : C(0);
        __syncwarp();
        if (lane == 0) {
          if (a.k > 0 && best >= 0)
            transfer_warp<C, NP>(st.dp, static_cast<C>((gi - best % a.nx) * a.step),
                                 static_cast<C>((gj - best / a.nx) * a.step), st.p);
          else
            for (int c = 0; c < NP; ++c) st.p[c] = st.dp[c];
          st.q = q;
          st.win.w = 0;
          st.iters = 0;
          st.converged = 0;
          st.zncc = nan("");
          st.status = DIC_PT_MAX_ITER;
        }
      }
      if (lane == 0) st.item = item;
    }
    __syncthreads();
    if (st.item >= n_front) break;
    const int q = st.q;
    const int xc = r + (q % a.nx) * a.step, yc = r + (q / a.nx) * a.step;

    // ---- 2. reference subset: its gray tile and the reference coefficients
    //         around it, staged in shared memory (TMA where the planes allow)
    const int rx0 = xc - r - 1, ry0 = yc - r - 1;                  // coefficient window origin
    const int rxa = rx0 - (((rx0 % XALIGN) + XALIGN) % XALIGN);    // TMA-aligned column
    const int gxa = (xc - r) - (((xc - r) * tl.gray_es) % 16) / tl.gray_es;   // gray tile column
    {
      if (tid == 0 && (tl.coef_tma || tl.gray_tma)) {
        fence_proxy_async_shared();
        uint32_t bytes = 0;
        if (tl.coef_tma) bytes += static_cast<uint32_t>(tl.bxc * tl.byc * sizeof(T));
        if (tl.gray_tma) bytes += static_cast<uint32_t>(tl.bxg * S * tl.gray_es);
        mbar_arrive_expect_tx(&s_bar, bytes);
        if (tl.coef_tma) tma_load_2d(s_win, &tm_cref, rxa, ry0, &s_bar);
        if (tl.gray_tma) tma_load_2d(s_gray, &tm_gray, gxa, yc - r, &s_bar);
      }
      if (!tl.coef_tma) {
        for (int row = warp; row < S + 2; row += NW) {
          const int gy = mirror_near(ry0 + row, a.H);
          const T* src = a.c_ref + static_cast<int64_t>(gy) * a.ldc;
          T* dst = s_win + row * tl.bxc + (rx0 - rxa);
          for (int c = lane; c < S + 2; c += 32) dst[c] = src[mirror_near(rx0 + c, a.W)];
        }
      }
      if (!tl.gray_tma) {
        const int es = tl.gray_es;
        for (int row = warp; row < S; row += NW) {
          const unsigned char* src = static_cast<const unsigned char*>(a.ref_gray.data) +
                                     static_cast<int64_t>(yc - r + row) * a.ref_gray.stride +
                                     static_cast<int64_t>(gxa) * es;
          unsigned char* dst = s_gray + row * gpitch;
          for (int c = lane; c < (S + (xc - r - gxa)) * es; c += 32) dst[c] = src[c];
        }
      }
      if (tl.coef_tma || tl.gray_tma) {
        if (!tma_wait()) return;
      } else {
        __syncthreads();
      }
      // mirror the coefficient rows and columns that fall outside the image
      if (tl.coef_tma && (rx0 < 0 || ry0 < 0 || rx0 + S + 2 > a.W || ry0 + S + 2 > a.H)) {
        T* w0 = s_win + (rx0 - rxa);
        for (int e = tid; e < S + 2; e += NT) {
          if (rx0 < 0) w0[e * tl.bxc + 0] = w0[e * tl.bxc + 2];
          if (rx0 + S + 2 > a.W) w0[e * tl.bxc + S + 1] = w0[e * tl.bxc + S - 1];
        }
        __syncthreads();
        for (int e = tid; e < S + 2; e += NT) {
          if (ry0 < 0) w0[e] = w0[2 * tl.bxc + e];
          if (ry0 + S + 2 > a.H) w0[(S + 1) * tl.bxc + e] = w0[(S - 1) * tl.bxc + e];
        }
        __syncthreads();
      }
    }
    const unsigned char* gtile = s_gray + (xc - r - gxa) * tl.gray_es;   // column 0 of the subset
    if (tid == 0) st.f0 = tile_gray<C>(gtile, gpitch, gdt, r, r);
    {
      const T* wref = s_win + (rx0 - rxa);
      const T f0 = tile_gray<T>(gtile, gpitch, gdt, r, r);
      T A[3][M2 + 1], Bf[2][D + 1], Bs[2][D + 1];
      T sf = T(0), sff = T(0);
#pragma unroll
      for (int j = 0; j <= M2; ++j) A[0][j] = A[1][j] = A[2][j] = T(0);
#pragma unroll
      for (int j = 0; j <= D; ++j) Bf[0][j] = Bf[1][j] = Bs[0][j] = Bs[1][j] = T(0);
      // PACKM: the fx and fy terms of a moment summed as one packed pair,
      // A02[j] = (A[0][j], A[2][j]), Bf2[j] = (Bf[0][j], Bf[1][j]), Bs2[j] = (Bs[0][j], Bs[1][j])
      // (128-thread FP32 blocks of up to 6 parameters, where the registers allow it)
      constexpr bool PACKM = NT == 128 && NP <= 6 && sizeof(T) == 4;
      Pair<T> A02[M2 + 1], Bf2[D + 1], Bs2[D + 1];
#pragma unroll
      for (int j = 0; j <= M2; ++j) A02[j] = pair(T(0), T(0));
#pragma unroll
      for (int j = 0; j <= D; ++j) Bf2[j] = Bs2[j] = pair(T(0), T(0));
      // the column walk keeps the three coefficient rows around the pixel in
      // registers: each row loads only the row below
      T m0 = T(0), m1 = T(0), m2 = T(0), z0 = T(0), z2 = T(0);
      if (row0 < row1) {
        const T* cm = wref + row0 * tl.bxc + col;   // row above, column left
        m0 = cm[0];
        m1 = cm[1];
        m2 = cm[2];
        z0 = cm[tl.bxc];
        z2 = cm[tl.bxc + 2];
      }
      T z1 = row0 < row1 ? wref[(row0 + 1) * tl.bxc + col + 1] : T(0);
      // f - f0 of this thread's pixels, converted from the gray tile by one loop per
      // element type (the type is the same for every pixel)
      {
        T* fo = s_f + row0 * S + col;
        const unsigned char* gi = gtile + row0 * gpitch + col * tl.gray_es;
        auto conv = [&](auto load) {
          for (int row = row0; row < row1; ++row, fo += S, gi += gpitch) *fo = load(gi) - f0;
        };
        switch (gdt) {
          case DIC_U8:
            conv([](const unsigned char* g) { return tile_gray<T>(g, 0, DIC_U8, 0, 0); });
            break;
          case DIC_U16:
            conv([](const unsigned char* g) { return tile_gray<T>(g, 0, DIC_U16, 0, 0); });
            break;
          case DIC_BF16:
            conv([](const unsigned char* g) { return tile_gray<T>(g, 0, DIC_BF16, 0, 0); });
            break;
          case DIC_F32:
            conv([](const unsigned char* g) { return tile_gray<T>(g, 0, DIC_F32, 0, 0); });
            break;
          default:
            conv([](const unsigned char* g) { return tile_gray<T>(g, 0, DIC_F64, 0, 0); });
            break;
        }
      }
      if (tl.gray_alias) __syncthreads();   // every gray level read before the gradients overwrite them
      T dyv = static_cast<T>(row0 - r);   // dy of the row, counted in T (exact)
      for (int row = row0; row < row1; ++row) {
        const int pix = row * S + col;
        // exact derivative of the reference spline at the pixel:
        // (-1/2, 0, 1/2) along one axis times (1, 4, 1)/6 along the other
        const T* cp = wref + (row + 2) * tl.bxc + col;
        const T p0 = cp[0], p1 = cp[1], p2 = cp[2];
        // (bicubic convolution: the central difference (f[k+1] - f[k-1]) / 2)
        T fx, fy;
        if (GEN && keys) {
          fx = (z2 - z0) * T(0.5);
          fy = (p1 - m1) * T(0.5);
        } else {
          fx = ((m2 - m0) + T(4) * (z2 - z0) + (p2 - p0)) * (T(1) / T(12));
          fy = ((p0 - m0) + T(4) * (p1 - m1) + (p2 - m2)) * (T(1) / T(12));
        }
        m0 = z0;
        m1 = z1;
        m2 = z2;
        z0 = p0;
        z1 = p1;
        z2 = p2;
        s_fg[pix] = pair(fx, fy);
        const T fp = s_f[pix];
        sf += fp;
        sff += fp * fp;
        T dyp[M2 + 1];
        dyp[0] = T(1);
#pragma unroll
        for (int j = 1; j <= M2; ++j) dyp[j] = dyp[j - 1] * dyv;
        dyv += T(1);
        if constexpr (PACKM) {
          const Pair<T> fg = pair(fx, fy);
          const Pair<T> w2 = pmul(fg, fg);                // (fx^2, fy^2)
          const Pair<T> fb = pmul(fg, pair(fp, fp));      // (fx f', fy f')
          const T wxy = fx * fy;
          A02[0] = padd(A02[0], w2);
          A[1][0] += wxy;
#pragma unroll
          for (int j = 1; j <= M2; ++j) {
            A02[j] = pfma(w2, pair(dyp[j], dyp[j]), A02[j]);
            A[1][j] += wxy * dyp[j];
          }
          Bf2[0] = padd(Bf2[0], fb);
          Bs2[0] = padd(Bs2[0], fg);
#pragma unroll
          for (int j = 1; j <= D; ++j) {
            Bf2[j] = pfma(fb, pair(dyp[j], dyp[j]), Bf2[j]);
            Bs2[j] = pfma(fg, pair(dyp[j], dyp[j]), Bs2[j]);
          }
        } else {
          const T wxx = fx * fx, wxy = fx * fy, wyy = fy * fy;
#pragma unroll
          for (int j = 0; j <= M2; ++j) {
            A[0][j] += wxx * dyp[j];
            A[1][j] += wxy * dyp[j];
            A[2][j] += wyy * dyp[j];
          }
          const T fxb = fx * fp, fyb = fy * fp;
#pragma unroll
          for (int j = 0; j <= D; ++j) {
            Bf[0][j] += fxb * dyp[j];
            Bf[1][j] += fyb * dyp[j];
            Bs[0][j] += fx * dyp[j];
            Bs[1][j] += fy * dyp[j];
          }
        }
      }
      if constexpr (PACKM) {
#pragma unroll
        for (int j = 0; j <= M2; ++j) {
          A[0][j] = A02[j].x;
          A[2][j] = A02[j].y;
        }
#pragma unroll
        for (int j = 0; j <= D; ++j) {
          Bf[0][j] = Bf2[j].x;
          Bf[1][j] = Bf2[j].y;
          Bs[0][j] = Bs2[j].x;
          Bs[1][j] = Bs2[j].y;
        }
      }
#pragma unroll
      for (int tt = 0; tt < 3; ++tt) {
        T v[pow2ceil(NMOM)];
#pragma unroll
        for (int e = NMOM; e < pow2ceil(NMOM); ++e) v[e] = T(0);
#pragma unroll
        for (int j = 0; j <= M2; ++j)
#pragma unroll
          for (int i = 0; i + j <= M2; ++i) v[mono(i, j, M2)] = dxp[i] * A[tt][j];
        parts(v, tt * NMOM, NMOM);
      }
      {
        T v[pow2ceil(NP)], w[pow2ceil(NP)];
#pragma unroll
        for (int c = NP; c < pow2ceil(NP); ++c) v[c] = w[c] = T(0);
#pragma unroll
        for (int c = 0; c < NP; ++c) {
          v[c] = dxp[sd_i(c)] * Bf[sd_t(c)][sd_j(c)];
          w[c] = dxp[sd_i(c)] * Bs[sd_t(c)][sd_j(c)];
        }
        parts(v, 3 * NMOM, NP);
        parts(w, 3 * NMOM + NP, NP);
      }
      {
        T v[2] = {sf, sff};
        parts(v, 3 * NMOM + 2 * NP, 2);
      }
    }
    __syncthreads();
    if (warp == 0) {
      gather(NV_PRE);
      finish_reference<C, NP, NMOM, M2, ANYCOST, SC>(st, s_out, N, lane, a.cost);
      if constexpr (LM) {
        // the undamped Hessian, kept for the damped inverses of every iteration
        for (int e = lane; e < NP * NP; e += 32) {
          const int ca = e / NP, cb = e % NP;
          lms.H[e] = s_out[(sd_t(ca) + sd_t(cb)) * NMOM + mono(sd_i(ca) + sd_i(cb), sd_j(ca) + sd_j(cb), M2)];
        }
        for (int e = lane; e < NP * NP; e += 32) lms.X0[e] = st.sv.X[e];
        if (lane == 0) {
          lms.lam = C(kLmLambda0);
          lms.has_best = 0;
        }
      }
      if (lane == 0) {
        if (st.ctl == 0)
          plan_window<C, NP>(st, xc, yc, r, a.W, a.H, tl, XALIGN);
        else
          st.status = st.ctl == 3 ? DIC_PT_FLAT : DIC_PT_SINGULAR;
      }
    }
    __syncthreads();

    // ---- 3. IC-GN iterations, then 4. the final ZNCC pass
    const T xlo = static_cast<T>(1 - xc), xhi = static_cast<T>(a.W - 2 - xc);
    const T ylo = static_cast<T>(1 - yc), yhi = static_cast<T>(a.H - 2 - yc);
    const C thr2 = static_cast<C>(a.conv_threshold * a.conv_threshold);
    bool running = st.ctl == 0;
    bool final_pass = false;
    while (running) {
      // stage the window that lane 0 planned (st is only written between barriers)
      const int stage = st.stage;
      const Window w = (stage == 1 || stage == 3) ? st.next : st.win;
      if (stage == 1) {
        if (tid == 0) {
          fence_proxy_async_shared();
          mbar_arrive_expect_tx(&s_bar, static_cast<uint32_t>(tl.bxc * tl.byc * sizeof(T)));
          tma_load_2d(s_win, &tm_cdef, w.x0, w.y0, &s_bar);
        }
        if (!tma_wait()) return;
      } else if (stage == 3) {
        for (int row = warp; row < w.h; row += NW) {
          const T* src = a.c_def + static_cast<int64_t>(w.y0 + row) * a.ldc + w.x0;
          T* dst = s_win + row * w.w;
          for (int c = lane; c < w.w; c += 32) dst[c] = src[c];
        }
        __syncthreads();
      }
      const T* pw = st.p;
      T ax = pw[0] + dxv, ay = pw[1], bx = T(0), by = T(1), cxq = T(0), cyq = T(0);
      if (NP >= 6) {
        ax += pw[2] * dxv;
        ay += pw[4] * dxv;
        bx = pw[3];
        by = T(1) + pw[5];
      }
      if (NP >= 12) {
        ax += pw[6] * dxv * dxv;
        ay += pw[9] * dxv * dxv;
        bx += pw[7] * dxv;
        by += pw[10] * dxv;
        cxq = pw[8];
        cyq = pw[11];
      }
      const T f0 = st.f0;
      T acc[NACC];
#pragma unroll
      for (int e = 0; e < NACC; ++e) acc[e] = T(0);
      T bad = T(0);
      if (stage != 2) {
        const T* base = s_win + (yc - 1 - w.y0) * w.w + (xc - 1 - w.x0);
        sample_column<T, D, true, GEN>(base, w.w, ax, bx, cxq, ay, by, cyq, xlo, xhi, ylo, yhi, f0, row0, row1, r,
                                     S, col, s_f, s_fg, LM && final_pass, st.inside != 0, keys, acc, bad);
      } else {
        const T* base = a.c_def + static_cast<int64_t>(yc - 1) * a.ldc + (xc - 1);
        sample_column_global<T, D, true>(base, a.ldc, ax, bx, cxq, ay, by, cyq, xlo, xhi, ylo, yhi, f0, row0, row1,
                                       r, S, col, s_f, s_fg, LM && final_pass, GEN && keys, acc, bad);
      }
      if (!final_pass) {
        T v[pow2ceil(NV_IT)];
        v[0] = acc[0];
        v[1] = acc[1];
#pragma unroll
        for (int c = 0; c < NP; ++c) v[2 + c] = dxp[sd_i(c)] * acc[2 + sd_t(c) * (D + 1) + sd_j(c)];
        v[2 + NP] = bad;
        v[3 + NP] = acc[2 + 2 * (D + 1)];
#pragma unroll
        for (int e = NV_IT; e < pow2ceil(NV_IT); ++e) v[e] = T(0);
        parts(v, 0, NV_IT);
      } else {
        T v[4] = {acc[0], acc[1], acc[2], bad};
        parts(v, 0, NV_FIN);
      }
      __syncthreads();
      if (warp == 0) {
        gather(final_pass ? NV_FIN : NV_IT);
        if (lane == 0 && (st.stage == 1 || st.stage == 3)) st.win = st.next;
        if (!final_pass) {
          int ctl;
          if constexpr (LM)
            ctl = lm_update<C, NP>(st, lms, s_out, N, static_cast<C>(r), thr2, lane, a.cost);
          else
            ctl = gauss_newton_update<C, NP, ANYCOST, SC>(st, s_out, N, static_cast<C>(r), thr2, lane, a.cost);
          if (lane == 0) {
            if (ctl == 5) {
              st.status = DIC_PT_OUT_OF_BOUNDS;
              st.ctl = 5;
            } else if (ctl == 2) {
              st.status = DIC_PT_FLAT;
              st.ctl = 2;
            } else {
              st.iters += 1;
              if (ctl == 1) st.converged = 1;
              const bool done = ctl == 1 || st.iters >= a.max_iter;
              if (done && !LM) {
                // Gauss-Newton: the coefficient of this iteration's pass, which was in
                // bounds and not flat (the update tested both); p includes the update
                if constexpr (S64) {
                  // normalised in FP64 from the FP32 sums
                  const double sg = s_out[0], sgg = s_out[1], sfg = s_out[3 + NP];
                  const double nu = sg / static_cast<double>(N);
                  const double dg = sqrt(fmax(sgg - sg * nu, 0.0));
                  st.zncc = (sfg - st.mu64 * sg) / (st.delta_f64 * dg);
                } else {
                  const C sg = s_out[0], sgg = s_out[1], sfg = s_out[3 + NP];
                  const C nu = sg / static_cast<C>(N);
                  const C dg = sqrt(fmax(sgg - sg * nu, C(0)));
                  st.zncc = static_cast<double>((sfg - st.mu * sg) / (st.delta_f * dg));
                }
                if (!st.converged)
                  st.status = DIC_PT_MAX_ITER;
                else if (st.zncc < a.zncc_min)
                  st.status = DIC_PT_LOW_ZNCC;
                else
                  st.status = DIC_PT_OK;
                st.ctl = 7;
              } else {
                st.ctl = done ? 6 : 0;   // 6: Levenberg-Marquardt's final pass
                plan_window<C, NP>(st, xc, yc, r, a.W, a.H, tl, XALIGN);
              }
            }
          }
        } else if (lane == 0) {
          // normalisation of the final correlation coefficient in C (its sums are in C)
          const C sg = s_out[0], sgg = s_out[1], sfg = s_out[2];
          const C nu = sg / static_cast<C>(N);
          const C dg = sqrt(fmax(sgg - sg * nu, C(0)));
          if (s_out[3] > C(0.5)) {
            st.status = DIC_PT_OUT_OF_BOUNDS;
          } else if (is_flat<C>(dg, nu + st.f0, N)) {
            st.status = DIC_PT_FLAT;
          } else {
            // sum (f - f_m)(g - g_m) = sum f' g' - mu sum g'
            st.zncc = static_cast<double>((sfg - st.mu * sg) / (st.delta_f * dg));
            if (!st.converged)
              st.status = DIC_PT_MAX_ITER;
            else if (st.zncc < a.zncc_min)
              st.status = DIC_PT_LOW_ZNCC;
            else
              st.status = DIC_PT_OK;
          }
          st.ctl = 7;
        }
      }
      __syncthreads();
      const int ctl = st.ctl;
      if (ctl == 6) {
        final_pass = true;
      } else if (ctl != 0) {
        running = false;
      }
    }

    // ---- 5. results and claims (warp 1, while warp 0 sets up the next point; the
    //         named barrier of warps 0 and 1 orders warp 1's reads of st before
    //         warp 0 rewrites it)
    if (warp == 0) {
      named_barrier_sync(1, 64);
    } else if (warp == 1) {
      const int status = st.status;
      const double pv = lane < NP ? static_cast<double>(st.p[lane]) : 0.0;
      const float z = static_cast<float>(st.zncc);
      const int iters = st.iters, conv = st.converged;
      named_barrier_sync(1, 64);
      if (lane < NP) a.pts.p[static_cast<int64_t>(q) * NP + lane] = pv;
      if (lane == 0) a.pts.u[q] = pv;
      if (lane == 1) a.pts.v[q] = pv;
      if (lane == 2) {
        a.pts.zncc[q] = z;
        a.pts.accept[q] = status == DIC_PT_OK
                              ? (static_cast<int64_t>(a.k) << 32) |
                                    static_cast<int64_t>(static_cast<uint32_t>(__float_as_int(z)))
                              : -1;
      }
      if (lane == 3) {
        a.pts.iters[q] = iters;
        a.pts.converged[q] = static_cast<uint8_t>(conv);
        a.pts.status[q] = static_cast<uint8_t>(status);
      }
      if (status == DIC_PT_OK && lane < 4) {
        const int gi = q % a.nx, gj = q / a.nx;
        int nb = -1;
        if (lane == 0 && gi > 0) nb = q - 1;
        if (lane == 1 && gi < a.nx - 1) nb = q + 1;
        if (lane == 2 && gj > 0) nb = q - a.nx;
        if (lane == 3 && gj < a.ny - 1) nb = q + a.nx;
        if (nb >= 0 && (a.roi_ok == nullptr || a.roi_ok[nb]) &&
            atomicCAS(&a.pts.wave[nb], -1, a.k + 1) == -1) {
          const int pos = atomicAdd(&a.counters[kCount + nxt], 1);
          a.next[pos] = nb;
        }
      }
    }
  }
}

// Raises the kernel's dynamic shared-memory limit to the device's opt-in limit
// less its static shared memory, once per instantiation (thread-safe); the
// largest tile set (S = 61, FP64 coefficients, 8-byte gray) stays below it.
template <typename T, int NP, int NT, int MODE>
cudaError_t configure_wave_smem() {
  static const cudaError_t result = []() {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, wave_kernel<T, NP, NT, MODE>);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(wave_kernel<T, NP, NT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin - static_cast<int>(fa.sharedSizeBytes));
    return e;
  }();
  return result;
}

template <typename T, int NP, int NT, int MODE>
cudaError_t launch_wave_nt(const WaveArgs<T>& a, const CUtensorMap* maps, int grid, cudaStream_t s) {
  const size_t smem = static_cast<size_t>(a.tiles.smem_bytes);
  const cudaError_t configured = configure_wave_smem<T, NP, NT, MODE>();
  if (configured != cudaSuccess) return configured;
  wave_kernel<T, NP, NT, MODE><<<grid, NT, smem, s>>>(a, maps[0], maps[1], maps[2]);
  return cudaGetLastError();
}

template <typename T, int NP, int MODE>
cudaError_t launch_wave_mode(const WaveArgs<T>& a, const CUtensorMap* maps, int grid, cudaStream_t s) {
  return a.threads == kWaveThreadsSmall ? launch_wave_nt<T, NP, kWaveThreadsSmall, MODE>(a, maps, grid, s)
                                        : launch_wave_nt<T, NP, kWaveThreads, MODE>(a, maps, grid, s);
}

template <typename T, int NP, int NT, int MODE>
int blocks_per_sm_nt(size_t smem) {
  if (configure_wave_smem<T, NP, NT, MODE>() != cudaSuccess) return 1;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, wave_kernel<T, NP, NT, MODE>, NT, smem) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

}  // namespace

// one instantiation of the wave kernel: launch, and resident blocks per SM
template <typename T, int NP, int MODE>
cudaError_t launch_wave_inst(const WaveArgs<T>& a, const CUtensorMap* maps, int grid, cudaStream_t s);
template <typename T, int NP, int MODE>
int blocks_per_sm_inst(int threads, size_t smem);

}  // namespace dic
