// One propagation wave: every point on the frontier is correlated by one block.
//
// Per point (Sec. 2.2, Eq. 4, Eq. 5; Sec. 2.4 for the propagation):
//   1. starting warp: the seed's integer offset (wave 0), else the warp of the
//      accepted 4-neighbour with the highest ZNCC, re-expanded about this centre;
//   2. reference subset: f, f - f_m and the exact spline gradient of the
//      reference at the S x S pixels, and the Gauss-Newton Hessian
//      H = sum SD^T SD of the steepest-descent images SD = grad f . dxi/dp,
//      assembled from gradient moments and factorised (Cholesky) in FP64;
//   3. inverse-compositional Gauss-Newton: sample the deformed spline at the
//      warped pixels, reduce sum g, sum g^2 and sum SD g, solve
//      dp = -H^-1 sum SD (f - f_m - (df/dg)(g - g_m)) in FP64, update
//      p <- p o dp^-1, stop when ||dp|| < threshold;
//   4. ZNCC = sum (f - f_m)(g - g_m) / (df dg) at the final p; accept when
//      converged, in bounds and ZNCC >= cut-off;
//   5. an accepted point claims its unvisited in-ROI 4-neighbours for the next wave.
//
// Threads map to pixels by column: thread t < S * bands owns column t % S and
// the rows of band t / S. The deformed coefficients around the warped subset are
// staged in shared memory once and re-staged only when the subset leaves them.
#include <math.h>

#include "dic_internal.cuh"

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

template <typename T>
__device__ __forceinline__ int floor_int(T x);
template <>
__device__ __forceinline__ int floor_int<float>(float x) { return __float2int_rd(x); }
template <>
__device__ __forceinline__ int floor_int<double>(double x) { return __double2int_rd(x); }

// Cholesky of the SPD n x n matrix in A (row-major), L written to L.
// Returns false when a pivot is <= 1e-12 * max diagonal.
template <int N>
__device__ bool cholesky(const double* A, double* L) {
  double dmax = 0.0;
  for (int k = 0; k < N; ++k) dmax = fmax(dmax, fabs(A[k * N + k]));
  const double tol = 1e-12 * dmax;
  for (int k = 0; k < N; ++k) {
    double d = A[k * N + k];
    for (int m = 0; m < k; ++m) d -= L[k * N + m] * L[k * N + m];
    if (!(d > tol)) return false;
    const double lkk = sqrt(d);
    L[k * N + k] = lkk;
    for (int i = k + 1; i < N; ++i) {
      double s = A[i * N + k];
      for (int m = 0; m < k; ++m) s -= L[i * N + m] * L[k * N + m];
      L[i * N + k] = s / lkk;
    }
  }
  return true;
}

template <int N>
__device__ void cholesky_solve(const double* L, const double* b, double* x) {
  double y[N];
  for (int i = 0; i < N; ++i) {
    double s = b[i];
    for (int m = 0; m < i; ++m) s -= L[i * N + m] * y[m];
    y[i] = s / L[i * N + i];
  }
  for (int i = N - 1; i >= 0; --i) {
    double s = y[i];
    for (int m = i + 1; m < N; ++m) s -= L[m * N + i] * x[m];
    x[i] = s / L[i * N + i];
  }
}

// Solves A^T Z^T = R^T for two right-hand rows (6 x 6, partial pivoting), i.e. Z = R A^-1.
__device__ void rows_times_inverse6(const double (&A)[6][6], double (&R)[2][6]) {
  double M[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) M[i][j] = A[j][i];  // transpose
  double B[6][2];
  for (int i = 0; i < 6; ++i) {
    B[i][0] = R[0][i];
    B[i][1] = R[1][i];
  }
  for (int k = 0; k < 6; ++k) {
    int piv = k;
    for (int i = k + 1; i < 6; ++i)
      if (fabs(M[i][k]) > fabs(M[piv][k])) piv = i;
    if (piv != k) {
      for (int j = 0; j < 6; ++j) {
        double t = M[k][j];
        M[k][j] = M[piv][j];
        M[piv][j] = t;
      }
      for (int j = 0; j < 2; ++j) {
        double t = B[k][j];
        B[k][j] = B[piv][j];
        B[piv][j] = t;
      }
    }
    for (int i = k + 1; i < 6; ++i) {
      const double f = M[i][k] / M[k][k];
      for (int j = k; j < 6; ++j) M[i][j] -= f * M[k][j];
      B[i][0] -= f * B[k][0];
      B[i][1] -= f * B[k][1];
    }
  }
  for (int c = 0; c < 2; ++c)
    for (int i = 5; i >= 0; --i) {
      double s = B[i][c];
      for (int j = i + 1; j < 6; ++j) s -= M[i][j] * R[c][j];
      R[c][i] = s / M[i][i];
    }
}

// Monomial map of the quadratic warp: m(W(x; p)) ~= A(p) m(x) with
// m = [x^2, xy, y^2, x, y, 1], terms above second order dropped.
__device__ void quad_monomial_matrix(const double* p, double (&A)[6][6]) {
  const double p0 = p[0], p1 = p[1], a = 1.0 + p[2], b = p[3], c = p[4], d = 1.0 + p[5];
  const double q6 = p[6], q7 = p[7], q8 = p[8], q9 = p[9], q10 = p[10], q11 = p[11];
  // x'^2
  A[0][0] = a * a + 2.0 * p0 * q6;
  A[0][1] = 2.0 * a * b + 2.0 * p0 * q7;
  A[0][2] = b * b + 2.0 * p0 * q8;
  A[0][3] = 2.0 * p0 * a;
  A[0][4] = 2.0 * p0 * b;
  A[0][5] = p0 * p0;
  // x'y'
  A[1][0] = a * c + p0 * q9 + p1 * q6;
  A[1][1] = a * d + b * c + p0 * q10 + p1 * q7;
  A[1][2] = b * d + p0 * q11 + p1 * q8;
  A[1][3] = p0 * c + p1 * a;
  A[1][4] = p0 * d + p1 * b;
  A[1][5] = p0 * p1;
  // y'^2
  A[2][0] = c * c + 2.0 * p1 * q9;
  A[2][1] = 2.0 * c * d + 2.0 * p1 * q10;
  A[2][2] = d * d + 2.0 * p1 * q11;
  A[2][3] = 2.0 * p1 * c;
  A[2][4] = 2.0 * p1 * d;
  A[2][5] = p1 * p1;
  // x', y', 1
  A[3][0] = q6; A[3][1] = q7; A[3][2] = q8; A[3][3] = a; A[3][4] = b; A[3][5] = p0;
  A[4][0] = q9; A[4][1] = q10; A[4][2] = q11; A[4][3] = c; A[4][4] = d; A[4][5] = p1;
  A[5][0] = 0.0; A[5][1] = 0.0; A[5][2] = 0.0; A[5][3] = 0.0; A[5][4] = 0.0; A[5][5] = 1.0;
}

// p <- W(W^-1(.; dp); p). Rigid and affine are exact; quadratic takes the x' and
// y' rows of A(p) A(dp)^-1 (second-order monomial representation of the warps).
template <int NP>
__device__ void compose_inverse(double* p, const double* dp) {
  if (NP == 2) {
    p[0] -= dp[0];
    p[1] -= dp[1];
  } else if (NP == 6) {
    const double a = 1.0 + dp[2], b = dp[3], c = dp[4], d = 1.0 + dp[5];
    const double det = a * d - b * c;
    const double ia = d / det, ib = -b / det, ic = -c / det, id = a / det;
    const double it0 = -(ia * dp[0] + ib * dp[1]), it1 = -(ic * dp[0] + id * dp[1]);
    const double A = 1.0 + p[2], B = p[3], C = p[4], Dd = 1.0 + p[5];
    const double n00 = A * ia + B * ic, n01 = A * ib + B * id;
    const double n10 = C * ia + Dd * ic, n11 = C * ib + Dd * id;
    const double t0 = A * it0 + B * it1 + p[0], t1 = C * it0 + Dd * it1 + p[1];
    p[0] = t0;
    p[1] = t1;
    p[2] = n00 - 1.0;
    p[3] = n01;
    p[4] = n10;
    p[5] = n11 - 1.0;
  } else {
    double Ap[6][6], Ad[6][6];
    quad_monomial_matrix(p, Ap);
    quad_monomial_matrix(dp, Ad);
    double R[2][6];
    for (int j = 0; j < 6; ++j) {
      R[0][j] = Ap[3][j];
      R[1][j] = Ap[4][j];
    }
    rows_times_inverse6(Ad, R);
    p[6] = R[0][0]; p[7] = R[0][1]; p[8] = R[0][2]; p[2] = R[0][3] - 1.0; p[3] = R[0][4]; p[0] = R[0][5];
    p[9] = R[1][0]; p[10] = R[1][1]; p[11] = R[1][2]; p[4] = R[1][3]; p[5] = R[1][4] - 1.0; p[1] = R[1][5];
  }
}

// neighbour warp re-expanded about a centre offset (ddx, ddy) from it
template <int NP>
__device__ void transfer_warp(const double* pn, double ddx, double ddy, double* p) {
  for (int c = 0; c < NP; ++c) p[c] = pn[c];
  if (NP >= 6) {
    p[0] = pn[0] + pn[2] * ddx + pn[3] * ddy;
    p[1] = pn[1] + pn[4] * ddx + pn[5] * ddy;
  }
  if (NP >= 12) {
    p[0] += pn[6] * ddx * ddx + pn[7] * ddx * ddy + pn[8] * ddy * ddy;
    p[1] += pn[9] * ddx * ddx + pn[10] * ddx * ddy + pn[11] * ddy * ddy;
    p[2] = pn[2] + 2.0 * pn[6] * ddx + pn[7] * ddy;
    p[3] = pn[3] + pn[7] * ddx + 2.0 * pn[8] * ddy;
    p[4] = pn[4] + 2.0 * pn[9] * ddx + pn[10] * ddy;
    p[5] = pn[5] + pn[10] * ddx + 2.0 * pn[11] * ddy;
  }
}

template <int NP>
__device__ double update_norm(const double* dp, double r) {
  double s = dp[0] * dp[0] + dp[1] * dp[1];
  if (NP >= 6) s += r * r * (dp[2] * dp[2] + dp[3] * dp[3] + dp[4] * dp[4] + dp[5] * dp[5]);
  if (NP >= 12) {
    double q = 0.0;
    for (int c = 6; c < 12; ++c) q += dp[c] * dp[c];
    s += r * r * r * r * q;
  }
  return sqrt(s);
}

__device__ __forceinline__ bool is_flat(double delta, double mean, int count) {
  return delta / sqrt(static_cast<double>(count)) <= 1e-6 * fmax(fabs(mean), 1.0);
}

struct Window {
  int x0, y0, w, h;
};

template <typename T, int NP>
__global__ void __launch_bounds__(kThreads, 2) wave_kernel(WaveArgs<T> a) {
  constexpr int D = Shape<NP>::D;
  constexpr int M2 = 2 * D;
  constexpr int NMOM = (M2 + 1) * (M2 + 2) / 2;
  constexpr int NV_PRE = 3 * NMOM + 2 * NP + 2;  // H moments, sum SD fbar, sum SD, sum fbar^2, sum fbar
  constexpr int NV_IT = 2 + NP;                  // sum g', sum g'^2, sum SD g'

  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int S = a.S, r = a.r, N = S * S;
  const int SS = (N + 3) & ~3;
  T* s_fbar = reinterpret_cast<T*>(smem_raw);
  T* s_fx = s_fbar + SS;
  T* s_fy = s_fx + SS;
  T* s_win = s_fy + SS;

  __shared__ double s_red[kWarps * NV_PRE];
  __shared__ double s_out[NV_PRE];
  __shared__ double s_p[kMaxParams];
  __shared__ double s_L[NP * NP];
  __shared__ double s_sdf[NP], s_sds[NP];
  __shared__ double s_fm, s_df, s_sumfbar;
  __shared__ int s_item, s_ctl;
  __shared__ Window s_win_box;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cur = a.k % 3, nxt = (a.k + 1) % 3, old = (a.k + 2) % 3;
  if (blockIdx.x == 0 && tid == 0) {
    a.counters[kCount + old] = 0;
    a.counters[kWork + nxt] = 0;
    a.wave_sizes[a.k] = a.counters[kCount + cur];
  }
  const int n_front = a.counters[kCount + cur];

  // this thread's pixels
  const int col = tid % S;
  const int band = tid / S;
  const int row0 = band < a.bands ? band * a.band_h : S;
  const int row1 = min(row0 + a.band_h, S);
  const T dxv = static_cast<T>(col - r);
  T dxp[M2 + 1];
  dxp[0] = T(1);
#pragma unroll
  for (int i = 1; i <= M2; ++i) dxp[i] = dxp[i - 1] * dxv;

  // block-wide sum of per-thread values, written to s_out[0..NV) in FP64
  auto reduce_store = [&](int idx, int nv, T v) {
    v = warp_sum(v);
    if (lane == 0) s_red[warp * nv + idx] = static_cast<double>(v);
  };
  auto reduce_finish = [&](int nv) {
    __syncthreads();
    for (int i = tid; i < nv; i += kThreads) {
      double s = 0.0;
      for (int w = 0; w < kWarps; ++w) s += s_red[w * nv + i];
      s_out[i] = s;
    }
    __syncthreads();
  };

  for (;;) {
    if (tid == 0) s_item = atomicAdd(&a.counters[kWork + cur], 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= n_front) break;
    const int q = a.cur[item];
    const int gi = q % a.nx, gj = q / a.nx;
    const int xc = r + gi * a.step, yc = r + gj * a.step;

    // ---- 1. starting warp
    if (tid == 0) {
      double p[kMaxParams];
      if (a.k == 0) {
        for (int c = 0; c < NP; ++c) p[c] = a.pts.p[static_cast<int64_t>(q) * NP + c];
      } else {
        int best = -1;
        double bz = 0.0;
        int nbs[4] = {gi > 0 ? q - 1 : -1, gi < a.nx - 1 ? q + 1 : -1, gj > 0 ? q - a.nx : -1,
                      gj < a.ny - 1 ? q + a.nx : -1};
        for (int m = 0; m < 4; ++m) {
          const int nb = nbs[m];
          if (nb < 0) continue;
          const int wv = a.pts.wave[nb];
          if (wv < 0 || wv >= a.k || a.pts.status[nb] != DIC_PT_OK) continue;
          const double z = a.pts.zncc64[nb];
          if (best < 0 || z > bz || (z == bz && nb < best)) {
            best = nb;
            bz = z;
          }
        }
        if (best >= 0) {
          const int bi = best % a.nx, bj = best / a.nx;
          transfer_warp<NP>(a.pts.p + static_cast<int64_t>(best) * NP,
                            static_cast<double>((gi - bi) * a.step),
                            static_cast<double>((gj - bj) * a.step), p);
        } else {
          for (int c = 0; c < NP; ++c) p[c] = 0.0;
        }
      }
      for (int c = 0; c < NP; ++c) s_p[c] = p[c];
      s_win_box.w = 0;  // no window staged yet
    }

    // ---- 2. reference subset: gray levels and spline gradients
    T sf = T(0);
    for (int row = row0; row < row1; ++row) {
      const int64_t x = xc + col - r, y = yc + row - r;
      const int pix = row * S + col;
      const T f = load_gray<T>(a.ref_gray, x, y);
      s_fbar[pix] = f;
      sf += f;
      const int64_t xm = x > 0 ? x - 1 : 1, xp = x < a.W - 1 ? x + 1 : a.W - 2;
      const int64_t ym = y > 0 ? y - 1 : 1, yp = y < a.H - 1 ? y + 1 : a.H - 2;
      const T* cm = a.c_ref + ym * a.ldc;
      const T* c0 = a.c_ref + y * a.ldc;
      const T* cp = a.c_ref + yp * a.ldc;
      // exact derivative of the reference spline at the pixel: (-1/2, 0, 1/2) (x) (1, 4, 1)/6
      const T gxm = cm[xp] - cm[xm], gx0 = c0[xp] - c0[xm], gxp = cp[xp] - cp[xm];
      const T gym = cp[xm] - cm[xm], gy0 = cp[x] - cm[x], gyp = cp[xp] - cm[xp];
      s_fx[pix] = (gxm + T(4) * gx0 + gxp) * (T(1) / T(12));
      s_fy[pix] = (gym + T(4) * gy0 + gyp) * (T(1) / T(12));
    }
    reduce_store(0, 1, sf);
    reduce_finish(1);
    if (tid == 0) s_fm = s_out[0] / N;
    __syncthreads();
    const double fm = s_fm;

    T A[3][M2 + 1], Bf[2][D + 1], Bs[2][D + 1];
    T sfb2 = T(0), sfb = T(0);
#pragma unroll
    for (int j = 0; j <= M2; ++j) A[0][j] = A[1][j] = A[2][j] = T(0);
#pragma unroll
    for (int j = 0; j <= D; ++j) Bf[0][j] = Bf[1][j] = Bs[0][j] = Bs[1][j] = T(0);
    for (int row = row0; row < row1; ++row) {
      const int pix = row * S + col;
      const T fb = static_cast<T>(static_cast<double>(s_fbar[pix]) - fm);
      s_fbar[pix] = fb;
      const T fx = s_fx[pix], fy = s_fy[pix];
      const T dyv = static_cast<T>(row - r);
      T dyp[M2 + 1];
      dyp[0] = T(1);
#pragma unroll
      for (int j = 1; j <= M2; ++j) dyp[j] = dyp[j - 1] * dyv;
      const T wxx = fx * fx, wxy = fx * fy, wyy = fy * fy;
#pragma unroll
      for (int j = 0; j <= M2; ++j) {
        A[0][j] += wxx * dyp[j];
        A[1][j] += wxy * dyp[j];
        A[2][j] += wyy * dyp[j];
      }
      const T fxb = fx * fb, fyb = fy * fb;
#pragma unroll
      for (int j = 0; j <= D; ++j) {
        Bf[0][j] += fxb * dyp[j];
        Bf[1][j] += fyb * dyp[j];
        Bs[0][j] += fx * dyp[j];
        Bs[1][j] += fy * dyp[j];
      }
      sfb2 += fb * fb;
      sfb += fb;
    }
#pragma unroll
    for (int tt = 0; tt < 3; ++tt)
#pragma unroll
      for (int j = 0; j <= M2; ++j)
#pragma unroll
        for (int i = 0; i + j <= M2; ++i) reduce_store(tt * NMOM + mono(i, j, M2), NV_PRE, dxp[i] * A[tt][j]);
#pragma unroll
    for (int c = 0; c < NP; ++c) {
      reduce_store(3 * NMOM + c, NV_PRE, dxp[sd_i(c)] * Bf[sd_t(c)][sd_j(c)]);
      reduce_store(3 * NMOM + NP + c, NV_PRE, dxp[sd_i(c)] * Bs[sd_t(c)][sd_j(c)]);
    }
    reduce_store(3 * NMOM + 2 * NP, NV_PRE, sfb2);
    reduce_store(3 * NMOM + 2 * NP + 1, NV_PRE, sfb);
    reduce_finish(NV_PRE);

    if (tid == 0) {
      int ctl = 0;
      s_df = sqrt(fmax(s_out[3 * NMOM + 2 * NP], 0.0));
      s_sumfbar = s_out[3 * NMOM + 2 * NP + 1];
      if (is_flat(s_df, fm, N)) {
        ctl = 3;
      } else {
        double Hm[NP * NP];
        for (int ca = 0; ca < NP; ++ca)
          for (int cb = 0; cb < NP; ++cb) {
            const int tt = sd_t(ca) + sd_t(cb);
            Hm[ca * NP + cb] = s_out[tt * NMOM + mono(sd_i(ca) + sd_i(cb), sd_j(ca) + sd_j(cb), M2)];
          }
        if (!cholesky<NP>(Hm, s_L)) ctl = 4;
        for (int c = 0; c < NP; ++c) {
          s_sdf[c] = s_out[3 * NMOM + c];
          s_sds[c] = s_out[3 * NMOM + NP + c];
        }
      }
      s_ctl = ctl;
    }
    __syncthreads();

    // ---- 3. IC-GN iterations
    int status = DIC_PT_MAX_ITER;
    int iters = 0;
    bool converged = false;
    bool stopped = false;  // out of bounds or flat during the iterations
    double zncc = nan("");
    if (s_ctl == 3) {
      status = DIC_PT_FLAT;
      stopped = true;
    } else if (s_ctl == 4) {
      status = DIC_PT_SINGULAR;
      stopped = true;
    }
    const T fmT = static_cast<T>(fm);
    const T xlo = static_cast<T>(1 - xc), xhi = static_cast<T>(a.W - 2 - xc);
    const T ylo = static_cast<T>(1 - yc), yhi = static_cast<T>(a.H - 2 - yc);

    // Stage (if needed) the coefficients under the warped subset; returns whether
    // the shared window is usable (else samples read the global plane).
    auto stage_window = [&]() -> bool {
      double p[kMaxParams];
      for (int c = 0; c < NP; ++c) p[c] = s_p[c];
      double ex = 0.0, ey = 0.0;
      if (NP >= 6) {
        ex = r * (fabs(1.0 + p[2]) + fabs(p[3]));
        ey = r * (fabs(p[4]) + fabs(1.0 + p[5]));
      } else {
        ex = ey = r;
      }
      if (NP >= 12) {
        ex += static_cast<double>(r) * r * (fabs(p[6]) + fabs(p[7]) + fabs(p[8]));
        ey += static_cast<double>(r) * r * (fabs(p[9]) + fabs(p[10]) + fabs(p[11]));
      }
      ex += 0.01;
      ey += 0.01;
      const double cx = xc + p[0], cy = yc + p[1];
      if (!(fabs(p[0]) < 1e6 && fabs(p[1]) < 1e6 && ex < 1e6 && ey < 1e6)) return false;
      int nx0 = static_cast<int>(floor(cx - ex)) - 1, nx1 = static_cast<int>(floor(cx + ex)) + 2;
      int ny0 = static_cast<int>(floor(cy - ey)) - 1, ny1 = static_cast<int>(floor(cy + ey)) + 2;
      nx0 = max(nx0, 0);
      ny0 = max(ny0, 0);
      nx1 = min(nx1, a.W - 1);
      ny1 = min(ny1, a.H - 1);
      if (nx1 < nx0 || ny1 < ny0) return false;  // wholly outside: every sample is out of bounds
      const Window cw = s_win_box;
      if (cw.w > 0 && nx0 >= cw.x0 && ny0 >= cw.y0 && nx1 < cw.x0 + cw.w && ny1 < cw.y0 + cw.h)
        return true;
      constexpr int kMargin = 2;
      int wx0 = max(nx0 - kMargin, 0), wy0 = max(ny0 - kMargin, 0);
      int wx1 = min(nx1 + kMargin, a.W - 1), wy1 = min(ny1 + kMargin, a.H - 1);
      if (static_cast<int64_t>(wx1 - wx0 + 1) * (wy1 - wy0 + 1) > a.win_cap) {
        wx0 = nx0;
        wy0 = ny0;
        wx1 = nx1;
        wy1 = ny1;
        if (static_cast<int64_t>(wx1 - wx0 + 1) * (wy1 - wy0 + 1) > a.win_cap) return false;
      }
      const int ww = wx1 - wx0 + 1, wh = wy1 - wy0 + 1;
      __syncthreads();  // everyone has finished with the previous window
      for (int row = warp; row < wh; row += kWarps) {
        const T* src = a.c_def + static_cast<int64_t>(wy0 + row) * a.ldc + wx0;
        T* dst = s_win + row * ww;
        for (int c = lane; c < ww; c += 32) dst[c] = src[c];
      }
      if (tid == 0) s_win_box = Window{wx0, wy0, ww, wh};
      __syncthreads();
      return true;
    };

    // Sum over this thread's pixels at the current p. MODE 0: sum g', sum g'^2 and the
    // SD moments; MODE 1: sum g', sum g'^2, sum fbar g'. Returns false if a sample is
    // out of bounds.
    auto sample_pass = [&](int mode, T* acc) -> bool {
      const bool use_win = stage_window();
      const Window w = s_win_box;
      T p[kMaxParams];
      for (int c = 0; c < NP; ++c) p[c] = static_cast<T>(s_p[c]);
      // positions relative to the centre: x = ax + dy (bx + cxq dy), y = ay + dy (by + cyq dy)
      T ax = p[0] + dxv, ay = p[1], bx = T(0), by = T(1), cxq = T(0), cyq = T(0);
      if (NP >= 6) {
        ax += p[2] * dxv;
        ay += p[4] * dxv;
        bx = p[3];
        by = T(1) + p[5];
      }
      if (NP >= 12) {
        ax += p[6] * dxv * dxv;
        ay += p[9] * dxv * dxv;
        bx += p[7] * dxv;
        by += p[10] * dxv;
        cxq = p[8];
        cyq = p[11];
      }
      const int offx = xc - 1 - w.x0, offy = yc - 1 - w.y0;
      bool bad = false;
      for (int row = row0; row < row1; ++row) {
        const T dyv = static_cast<T>(row - r);
        const T xl = ax + dyv * (bx + cxq * dyv);
        const T yl = ay + dyv * (by + cyq * dyv);
        if (!(xl >= xlo && xl < xhi && yl >= ylo && yl < yhi)) {
          bad = true;
          continue;
        }
        const int ix = floor_int<T>(xl), iy = floor_int<T>(yl);
        const T tx = xl - static_cast<T>(ix), ty = yl - static_cast<T>(iy);
        T wx0, wx1, wx2, wx3, wy0, wy1, wy2, wy3;
        bspline_weights<T>(tx, wx0, wx1, wx2, wx3);
        bspline_weights<T>(ty, wy0, wy1, wy2, wy3);
        const T* b;
        int64_t ld;
        if (use_win) {
          b = s_win + (offy + iy) * w.w + (offx + ix);
          ld = w.w;
        } else {
          b = a.c_def + static_cast<int64_t>(yc + iy - 1) * a.ldc + (xc + ix - 1);
          ld = a.ldc;
        }
        const T r0 = wx0 * b[0] + wx1 * b[1] + wx2 * b[2] + wx3 * b[3];
        const T* b1 = b + ld;
        const T r1 = wx0 * b1[0] + wx1 * b1[1] + wx2 * b1[2] + wx3 * b1[3];
        const T* b2 = b1 + ld;
        const T r2 = wx0 * b2[0] + wx1 * b2[1] + wx2 * b2[2] + wx3 * b2[3];
        const T* b3 = b2 + ld;
        const T r3 = wx0 * b3[0] + wx1 * b3[1] + wx2 * b3[2] + wx3 * b3[3];
        const T g = wy0 * r0 + wy1 * r1 + wy2 * r2 + wy3 * r3;
        const T gp = g - fmT;
        const int pix = row * S + col;
        acc[0] += gp;
        acc[1] += gp * gp;
        if (mode == 0) {
          const T gx = gp * s_fx[pix], gy = gp * s_fy[pix];
          T dyp = T(1);
#pragma unroll
          for (int j = 0; j <= D; ++j) {
            acc[2 + j] += gx * dyp;
            acc[2 + D + 1 + j] += gy * dyp;
            dyp *= dyv;
          }
        } else {
          acc[2] += gp * s_fbar[pix];
        }
      }
      return !__syncthreads_or(bad);
    };

    if (!stopped) {
      for (int it = 0; it < a.max_iter; ++it) {
        T acc[2 + 2 * (D + 1)];
#pragma unroll
        for (int e = 0; e < 2 + 2 * (D + 1); ++e) acc[e] = T(0);
        if (!sample_pass(0, acc)) {
          status = DIC_PT_OUT_OF_BOUNDS;
          stopped = true;
          break;
        }
        reduce_store(0, NV_IT, acc[0]);
        reduce_store(1, NV_IT, acc[1]);
#pragma unroll
        for (int c = 0; c < NP; ++c)
          reduce_store(2 + c, NV_IT, dxp[sd_i(c)] * acc[2 + sd_t(c) * (D + 1) + sd_j(c)]);
        reduce_finish(NV_IT);
        if (tid == 0) {
          int ctl = 0;
          const double gm = s_out[0] / N;  // mean of g - f_m
          const double dg = sqrt(fmax(s_out[1] - N * gm * gm, 0.0));
          if (is_flat(dg, gm + static_cast<double>(fmT), N)) {
            ctl = 2;
          } else {
            const double ratio = s_df / dg;
            double b[NP], x[NP], dp[NP];
            for (int c = 0; c < NP; ++c) b[c] = s_sdf[c] - ratio * (s_out[2 + c] - gm * s_sds[c]);
            cholesky_solve<NP>(s_L, b, x);
            for (int c = 0; c < NP; ++c) dp[c] = -x[c];
            double p[kMaxParams];
            for (int c = 0; c < NP; ++c) p[c] = s_p[c];
            compose_inverse<NP>(p, dp);
            for (int c = 0; c < NP; ++c) s_p[c] = p[c];
            if (update_norm<NP>(dp, static_cast<double>(r)) < a.conv_threshold) ctl = 1;
          }
          s_ctl = ctl;
        }
        __syncthreads();
        const int ctl = s_ctl;
        if (ctl == 2) {
          status = DIC_PT_FLAT;
          stopped = true;
          break;
        }
        ++iters;
        if (ctl == 1) {
          converged = true;
          break;
        }
      }
    }

    // ---- 4. ZNCC at the final p, and the decision
    if (!stopped) {
      T acc[3] = {T(0), T(0), T(0)};
      if (!sample_pass(1, acc)) {
        status = DIC_PT_OUT_OF_BOUNDS;
      } else {
        reduce_store(0, 3, acc[0]);
        reduce_store(1, 3, acc[1]);
        reduce_store(2, 3, acc[2]);
        reduce_finish(3);
        const double gm = s_out[0] / N;
        const double dg = sqrt(fmax(s_out[1] - N * gm * gm, 0.0));
        if (is_flat(dg, gm + static_cast<double>(fmT), N)) {
          status = DIC_PT_FLAT;
        } else {
          zncc = (s_out[2] - gm * s_sumfbar) / (s_df * dg);
          if (!converged)
            status = DIC_PT_MAX_ITER;
          else if (zncc < a.zncc_min)
            status = DIC_PT_LOW_ZNCC;
          else
            status = DIC_PT_OK;
        }
      }
    }

    // ---- 5. results and claims
    if (tid == 0) {
      double* pq = a.pts.p + static_cast<int64_t>(q) * NP;
      for (int c = 0; c < NP; ++c) pq[c] = s_p[c];
      a.pts.u[q] = s_p[0];
      a.pts.v[q] = s_p[1];
      a.pts.zncc[q] = static_cast<float>(zncc);
      a.pts.zncc64[q] = zncc;
      a.pts.iters[q] = iters;
      a.pts.converged[q] = converged ? 1 : 0;
      a.pts.status[q] = static_cast<uint8_t>(status);
      if (status == DIC_PT_OK) {
        int nbs[4] = {gi > 0 ? q - 1 : -1, gi < a.nx - 1 ? q + 1 : -1, gj > 0 ? q - a.nx : -1,
                      gj < a.ny - 1 ? q + a.nx : -1};
        for (int m = 0; m < 4; ++m) {
          const int nb = nbs[m];
          if (nb < 0) continue;
          if (a.roi_ok && !a.roi_ok[nb]) continue;
          if (atomicCAS(&a.pts.wave[nb], -1, a.k + 1) == -1) {
            const int pos = atomicAdd(&a.counters[kCount + nxt], 1);
            a.next[pos] = nb;
          }
        }
      }
    }
    __syncthreads();
  }
}

__global__ void roi_flags_kernel(RoiArgs a) {
  const int64_t n = static_cast<int64_t>(a.nx) * a.ny;
  const int lane = threadIdx.x & 31;
  for (int64_t q = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; q < n;
       q += (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5) {
    const int xc = a.r + static_cast<int>(q % a.nx) * a.step;
    const int yc = a.r + static_cast<int>(q / a.nx) * a.step;
    bool all_in = true;
    for (int row = 0; row < a.S && all_in; ++row) {
      const uint8_t* m = static_cast<const uint8_t*>(a.mask.data) + (yc - a.r + row) * a.mask.stride;
      bool ok = true;
      for (int c = lane; c < a.S; c += 32) ok &= m[xc - a.r + c] != 0;
      all_in = __all_sync(0xffffffffu, ok);
    }
    if (lane == 0) a.roi_ok[q] = all_in ? 1 : 0;
  }
}

__global__ void reset_points_kernel(PointArrays pa, int nparams, const uint8_t* roi_ok) {
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < pa.n;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    pa.u[q] = 0.0;
    pa.v[q] = 0.0;
    for (int c = 0; c < nparams; ++c) pa.p[q * nparams + c] = 0.0;
    pa.zncc[q] = nanf("");
    pa.zncc64[q] = nan("");
    pa.iters[q] = 0;
    pa.converged[q] = 0;
    pa.status[q] = (roi_ok && !roi_ok[q]) ? DIC_PT_NOT_IN_ROI : DIC_PT_NOT_REACHED;
    pa.wave[q] = -1;
  }
}

__global__ void finalize_points_kernel(PointArrays pa, int nparams, int nan_rejected,
                                       int32_t* accepted) {
  int count = 0;
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < pa.n;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const bool ok = pa.status[q] == DIC_PT_OK;
    count += ok ? 1 : 0;
    if (nan_rejected && !ok) {
      const double nanv = nan("");
      pa.u[q] = nanv;
      pa.v[q] = nanv;
      for (int c = 0; c < nparams; ++c) pa.p[q * nparams + c] = nanv;
    }
  }
  count = warp_sum(count);
  if ((threadIdx.x & 31) == 0 && count) atomicAdd(accepted, count);
}

template <typename T, int NP>
cudaError_t launch_wave_np(const WaveArgs<T>& a, int grid, cudaStream_t s) {
  const size_t smem = wave_smem_bytes<T>(a.S, a.win_cap);
  static size_t configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(wave_kernel<T, NP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  wave_kernel<T, NP><<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int NP>
int blocks_per_sm_np(size_t smem) {
  cudaFuncSetAttribute(wave_kernel<T, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       static_cast<int>(smem));
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, wave_kernel<T, NP>, kThreads, smem) !=
      cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

}  // namespace

template <typename T>
size_t wave_smem_bytes(int S, int win_cap) {
  const size_t SS = (static_cast<size_t>(S) * S + 3) & ~static_cast<size_t>(3);
  return (3 * SS + static_cast<size_t>(win_cap)) * sizeof(T);
}

template <typename T>
cudaError_t launch_wave(const WaveArgs<T>& a, int nparams, int grid, cudaStream_t s) {
  switch (nparams) {
    case 2:
      return launch_wave_np<T, 2>(a, grid, s);
    case 6:
      return launch_wave_np<T, 6>(a, grid, s);
    default:
      return launch_wave_np<T, 12>(a, grid, s);
  }
}

template <typename T>
int wave_blocks_per_sm(int nparams, size_t smem) {
  switch (nparams) {
    case 2:
      return blocks_per_sm_np<T, 2>(smem);
    case 6:
      return blocks_per_sm_np<T, 6>(smem);
    default:
      return blocks_per_sm_np<T, 12>(smem);
  }
}

cudaError_t launch_roi_flags(const RoiArgs& a, cudaStream_t s) {
  const int64_t n = static_cast<int64_t>(a.nx) * a.ny;
  const int64_t blocks = (n * 32 + 255) / 256;
  roi_flags_kernel<<<static_cast<unsigned>(blocks < 65535 ? blocks : 65535), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_reset_points(const PointArrays& pa, int nparams, const uint8_t* roi_ok,
                                cudaStream_t s) {
  const int64_t blocks = (pa.n + 255) / 256;
  reset_points_kernel<<<static_cast<unsigned>(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(
      pa, nparams, roi_ok);
  return cudaGetLastError();
}

cudaError_t launch_finalize_points(const PointArrays& pa, int nparams, int nan_rejected,
                                   int32_t* accepted, cudaStream_t s) {
  const int64_t blocks = (pa.n + 255) / 256;
  finalize_points_kernel<<<static_cast<unsigned>(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(
      pa, nparams, nan_rejected, accepted);
  return cudaGetLastError();
}

template size_t wave_smem_bytes<float>(int, int);
template size_t wave_smem_bytes<double>(int, int);
template cudaError_t launch_wave<float>(const WaveArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_wave<double>(const WaveArgs<double>&, int, int, cudaStream_t);
template int wave_blocks_per_sm<float>(int, size_t);
template int wave_blocks_per_sm<double>(int, size_t);

}  // namespace dic
