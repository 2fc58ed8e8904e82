// Strain post-processing (Sec. 2.3): at every grid point the displacement gradient
// of a least-squares fit u = P c over the N x N window of grid points centred on it
// (Eq. 8-9; P = [1, x, y] or [1, x, y, x^2, y^2, x^2 y, x y^2, x^2 y^2]), the
// deformation gradient F = I + grad u (Eq. 6) and one of the five strain measures.
//
// Only accepted points (status 0) inside the grid enter a window, and the centre
// must be accepted. A full window (every point present) is the common case: there
// the odd-in-x basis terms {x, x y^2} are orthogonal to the others, so the fitted
// x slope is sum_ij i (a + b j^2) u_ij / s in grid units (i, j) with two constants
// a, b of the window, and the y slope sum_ij j (a + b i^2) u_ij / s, applied
// separably from shared-memory tiles. A window with missing points is fitted
// from its normal equations (grid units, unit-diagonal scaling, elimination
// without exchanges); a scaled pivot at or below 1e-5 leaves the point without
// strain (NaN). Arithmetic in FP32 on displacement offsets: from a reference point of
// the tile for the separable filter (whose slope weights sum to zero, so the reference
// drops out), from the centre, formed in FP64 and rounded once, for the general fit.
#include <math.h>

#include "dic_internal.cuh"

namespace dic {
namespace {

constexpr float kMinScaledPivot = 1e-5f;

// P(x, y) for the basis (Eq. 9, as printed)
__device__ __forceinline__ void basis_row(int basis, float x, float y, float* P) {
  P[0] = 1.0f;
  P[1] = x;
  P[2] = y;
  if (basis != DIC_STRAIN_BILINEAR) {
    P[3] = x * x;
    P[4] = y * y;
    P[5] = x * x * y;
    P[6] = x * y * y;
    P[7] = x * x * y * y;
  }
}

// General least squares over the valid points of the window (out of line: windows with
// missing points are the rare case) for a basis of K terms: returns NaN in .x when the
// design is not well posed; else the x and y slopes (grid units) of u and v. Which
// points are present comes from the block's staged offsets su (row pitch SX; NaN where
// a point is missing or outside the grid; centre at slot ec); the offsets from the
// centre are formed in FP64 from the staged displacements ud, vd and rounded once.
// Normal equations with
// unit-diagonal scaling, then elimination without exchanges, indexed at compile time
// (K fixed) so that the matrix lives in registers.
template <int K>
__device__ __noinline__ float4 fit_window(const StrainArgs& a, int h, const float* su, const double* ud,
                                          const double* vd, int SX, int ec, double uc, double vc) {
  const float4 fail = make_float4(__int_as_float(0x7fc00000), 0.0f, 0.0f, 0.0f);
  float M[K][K], ru[K], rv[K];
#pragma unroll
  for (int r = 0; r < K; ++r) {
    ru[r] = rv[r] = 0.0f;
#pragma unroll
    for (int c = 0; c < K; ++c) M[r][c] = 0.0f;
  }
  int count = 0;
  for (int dj = -h; dj <= h; ++dj) {
    for (int di = -h; di <= h; ++di) {
      const int e = ec + dj * SX + di;
      if (su[e] != su[e]) continue;                  // missing: not accepted, or outside the grid
      float P[8];
      basis_row(a.basis, static_cast<float>(di), static_cast<float>(dj), P);
      const float du = static_cast<float>(ud[e] - uc), dv = static_cast<float>(vd[e] - vc);
#pragma unroll
      for (int r = 0; r < K; ++r) {
        ru[r] += P[r] * du;
        rv[r] += P[r] * dv;
#pragma unroll
        for (int c = r; c < K; ++c) M[r][c] += P[r] * P[c];
      }
      ++count;
    }
  }
  if (count < K) return fail;
  float d[K];
#pragma unroll
  for (int r = 0; r < K; ++r) {
    if (!(M[r][r] > 0.0f)) return fail;
    d[r] = rsqrtf(M[r][r]);
  }
#pragma unroll
  for (int r = 0; r < K; ++r) {
#pragma unroll
    for (int c = r; c < K; ++c) M[r][c] *= d[r] * d[c];
#pragma unroll
    for (int c = 0; c < r; ++c) M[r][c] = M[c][r];
    ru[r] *= d[r];
    rv[r] *= d[r];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float piv = M[k][k];
    if (!(piv > kMinScaledPivot)) return fail;
    const float inv = 1.0f / piv;
#pragma unroll
    for (int r = k + 1; r < K; ++r) {
      const float f = M[r][k] * inv;
#pragma unroll
      for (int c = k + 1; c < K; ++c) M[r][c] -= f * M[k][c];
      ru[r] -= f * ru[k];
      rv[r] -= f * rv[k];
    }
  }
#pragma unroll
  for (int r = K - 1; r >= 0; --r) {
    float xu = ru[r], xv = rv[r];
#pragma unroll
    for (int c = r + 1; c < K; ++c) {
      xu -= M[r][c] * ru[c];
      xv -= M[r][c] * rv[c];
    }
    ru[r] = xu / M[r][r];
    rv[r] = xv / M[r][r];
  }
  // undo the scaling: coefficient r is d[r] z[r]
  return make_float4(d[1] * ru[1], d[2] * ru[2], d[1] * rv[1], d[2] * rv[2]);
}

// eigenvalues mu1 >= mu2 of the symmetric [[d11, d12], [d12, d22]]
__device__ __forceinline__ void sym_eig(float d11, float d12, float d22, float* mu1, float* mu2) {
  const float m = 0.5f * (d11 + d22);
  const float q = sqrtf(0.25f * (d11 - d22) * (d11 - d22) + d12 * d12);
  *mu1 = m + q;
  *mu2 = m - q;
}

// f(I + D) = m I + g (D - tr(D)/2 I) for a symmetric D with eigenvalues mu1, mu2,
// where m is the mean of f at 1 + mu_k and g their divided difference
__device__ __forceinline__ void spectral(float d11, float d12, float d22, float m, float g, float* e) {
  const float t = 0.5f * (d11 + d22);
  e[0] = m + g * (d11 - t);
  e[1] = m + g * (d22 - t);
  e[2] = g * d12;
}

// Sec. 2.3: strain (exx, eyy, exy) from H = grad u, formed from the small parts of
// F^T F = I + D or F F^T = I + D' so that no 1 is subtracted from a near-1 value.
__device__ __forceinline__ void strain_from_gradient(int measure, float h11, float h12, float h21, float h22,
                                                     float* e) {
  const bool left = measure == DIC_EULER_ALMANSI || measure == DIC_BIOT_LEFT;
  // D = H + H^T + H^T H (right) or D' = H + H^T + H H^T (left)
  const float d11 = left ? 2.0f * h11 + h11 * h11 + h12 * h12 : 2.0f * h11 + h11 * h11 + h21 * h21;
  const float d22 = left ? 2.0f * h22 + h21 * h21 + h22 * h22 : 2.0f * h22 + h12 * h12 + h22 * h22;
  const float d12 = left ? h12 + h21 + h11 * h21 + h12 * h22 : h12 + h21 + h11 * h12 + h21 * h22;
  if (measure == DIC_GREEN_LAGRANGE) {            // (F^T F - I) / 2
    e[0] = 0.5f * d11;
    e[1] = 0.5f * d22;
    e[2] = 0.5f * d12;
    return;
  }
  if (measure == DIC_EULER_ALMANSI) {             // (I - (F F^T)^-1) / 2 = (D' + det D' I) / (2 det(I + D'))
    const float det = d11 * d22 - d12 * d12;
    const float s = 0.5f / (1.0f + d11 + d22 + det);
    e[0] = (d11 + det) * s;
    e[1] = (d22 + det) * s;
    e[2] = d12 * s;
    return;
  }
  float mu1, mu2;
  sym_eig(d11, d12, d22, &mu1, &mu2);
  if (measure == DIC_HENCKY) {                    // ln sqrt(C): f(lambda) = ln(lambda) / 2
    const float m = 0.25f * (log1pf(mu1) + log1pf(mu2));
    const float z = (mu1 - mu2) / (1.0f + mu2);
    const float l = z < 1e-3f ? 1.0f - z * (0.5f - z * (1.0f / 3.0f)) : log1pf(z) / z;
    spectral(d11, d12, d22, m, 0.5f * l / (1.0f + mu2), e);
    return;
  }
  // Biot, right or left: sqrt(I + D) - I: f(lambda) = sqrt(lambda) - 1
  const float r1 = sqrtf(1.0f + mu1), r2 = sqrtf(1.0f + mu2);
  const float m = 0.5f * (mu1 / (1.0f + r1) + mu2 / (1.0f + r2));
  spectral(d11, d12, d22, m, 1.0f / (r1 + r2), e);
}

constexpr int kTileX = 32, kTileY = 16;   // grid points per block (one per thread; a warp per tile row)
// staged points per thread for a half-window h: kernels for h <= 4 (2 each) and for
// h <= 15, the largest window (6 each)
constexpr int staged_per_thread(int h) {
  return ((kTileX + 2 * h) * (kTileY + 2 * h) + kTileX * kTileY - 1) / (kTileX * kTileY);
}
constexpr int kSmallHalf = 4, kMaxHalf = 15;

// Block of kTileX x kTileY grid points. The block stages the displacements of its
// points and of a halo of h = (window - 1) / 2 points as FP32 offsets from one
// accepted point of the tile, the first in row-major order (points outside the grid
// or not accepted become NaN), and as the FP64 values (for the general fit), then
// applies the full-window slope filter separably:
// along each staged row the sums sum_i i d, sum_i d and sum_i i^2 d over the window's
// columns, then down each point's column the x slope sum_j (a + b j^2) (sum_i i d)_j
// and the y slope sum_j j (a (sum_i d)_j + b (sum_i i^2 d)_j). A NaN anywhere in a
// window reaches its sums (even through a zero weight), which sends the point to the
// general fit. Every load of a thread is issued before the first barrier; the
// reference point comes from one ballot per warp; three barriers in all.
template <int kStagedPerThread>
__global__ void __launch_bounds__(kTileX * kTileY, 2) strain_kernel(StrainArgs a) {
  extern __shared__ __align__(16) double smd[];
  const int h = (a.window - 1) / 2, N = a.window;
  const int SX = kTileX + 2 * h, SY = kTileY + 2 * h, NS = SX * SY;
  double* ud = smd;               // [SY][SX] staged displacements (for the general fit)
  double* vd = ud + NS;
  float* su = reinterpret_cast<float*>(vd + NS);   // [SY][SX] staged offsets of u
  float* sv = su + NS;            // ... of v
  float* fx = sv + NS;            // [2][SY][kTileX] row sums: sum i d   (u, v)
  float* f0 = fx + 2 * SY * kTileX;   // sum d
  float* f2 = f0 + 2 * SY * kTileX;   // sum i^2 d
  __shared__ int s_first[kTileY];     // per tile row: lane of its first accepted point, or 32
  __shared__ float2 s_ref[kTileY];    // ... and that point's (u, v) in FP32
  const int tid = threadIdx.x, tx = tid & (kTileX - 1), ty = tid / kTileX;
  const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;
  const int ic = x0 + tx, jc = y0 + ty;
  const bool inside = ic < a.nx && jc < a.ny;
  const int64_t q = static_cast<int64_t>(jc) * a.nx + ic;
  uint8_t st_c = 1;
  double uc = 0.0, vc = 0.0;
  if (inside) {
    st_c = a.status[q];
    uc = a.u[q];
    vc = a.v[q];
  }
  // the staged points of this thread: status and displacements, loaded now
  uint8_t sst[kStagedPerThread];
  double suq[kStagedPerThread], svq[kStagedPerThread];
#pragma unroll
  for (int k = 0; k < kStagedPerThread; ++k) {
    const int e = tid + k * kTileX * kTileY;
    sst[k] = 1;
    suq[k] = svq[k] = 0.0;
    if (e < NS) {
      const int i = x0 - h + e % SX, j = y0 - h + e / SX;
      if (i >= 0 && i < a.nx && j >= 0 && j < a.ny) {
        const int64_t qs = static_cast<int64_t>(j) * a.nx + i;
        sst[k] = a.status[qs];
        suq[k] = a.u[qs];
        svq[k] = a.v[qs];
      }
    }
  }
  // the tile's reference: the first accepted point in row-major order
  const unsigned acc = __ballot_sync(0xffffffffu, inside && st_c == 0);
  const int first = acc ? __ffs(acc) - 1 : kTileX;
  if (tx == 0) s_first[ty] = first;
  if (tx == first) s_ref[ty] = make_float2(static_cast<float>(uc), static_cast<float>(vc));
  __syncthreads();
  float2 ref = make_float2(0.0f, 0.0f);
  for (int r = 0; r < kTileY; ++r) {
    if (s_first[r] < kTileX) {
      ref = s_ref[r];
      break;
    }
  }
  // offsets are formed in FP32 after one conversion per value (FP64 arithmetic runs at a
  // small fraction of the FP32 rate here); exact when the displacements are FP32 values,
  // as the mixed path produces them
  const float nan_ = __int_as_float(0x7fc00000);
#pragma unroll
  for (int k = 0; k < kStagedPerThread; ++k) {
    const int e = tid + k * kTileX * kTileY;
    if (e < NS) {
      const bool ok = sst[k] == 0;
      su[e] = ok ? static_cast<float>(suq[k]) - ref.x : nan_;
      sv[e] = ok ? static_cast<float>(svq[k]) - ref.y : nan_;
      ud[e] = suq[k];
      vd[e] = svq[k];
    }
  }
  __syncthreads();
  for (int e = tid; e < 2 * SY * kTileX; e += blockDim.x) {
    const int comp = e >= SY * kTileX, rc = e - comp * SY * kTileX;
    const int row = rc / kTileX, c = rc & (kTileX - 1);
    const float* src = (comp == 0 ? su : sv) + row * SX + c;   // window columns c .. c + 2h
    float sx = 0.0f, s0 = 0.0f, s2 = 0.0f;
    float di = static_cast<float>(-h);                 // k - h, counted in FP32 (exact)
    for (int k = 0; k < N; ++k, di += 1.0f) {
      const float d = src[k];
      sx += di * d;
      s0 += d;
      s2 += di * di * d;
    }
    fx[e] = sx;
    f0[e] = s0;
    f2[e] = s2;
  }
  __syncthreads();
  if (!inside) return;
  float4 g = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  bool ok = st_c == 0;
  if (ok) {
    float sux = 0.0f, suy = 0.0f, svx = 0.0f, svy = 0.0f;
    const int o = ty * kTileX + tx, ov = SY * kTileX;
    float dj = static_cast<float>(-h);                 // k - h, counted in FP32 (exact)
    for (int k = 0; k < N; ++k, dj += 1.0f) {
      const float wxj = a.wa + a.wb * dj * dj;
      const int r = o + k * kTileX;
      sux += wxj * fx[r];
      svx += wxj * fx[ov + r];
      suy += dj * (a.wa * f0[r] + a.wb * f2[r]);
      svy += dj * (a.wa * f0[ov + r] + a.wb * f2[ov + r]);
    }
    if (isfinite(sux) && isfinite(suy) && isfinite(svx) && isfinite(svy)) {
      g = make_float4(sux, suy, svx, svy);
    } else {
      const int ec = (ty + h) * SX + tx + h;
      g = a.basis == DIC_STRAIN_BILINEAR ? fit_window<3>(a, h, su, ud, vd, SX, ec, uc, vc)
                                         : fit_window<8>(a, h, su, ud, vd, SX, ec, uc, vc);
      ok = g.x == g.x;
    }
  }
  if (ok) {
    const float inv_s = 1.0f / static_cast<float>(a.step);   // grid units -> pixels
    const float h11 = g.x * inv_s, h12 = g.y * inv_s, h21 = g.z * inv_s, h22 = g.w * inv_s;
    float e[3];
    strain_from_gradient(a.measure, h11, h12, h21, h22, e);
    a.dudx[q] = h11;
    a.dudy[q] = h12;
    a.dvdx[q] = h21;
    a.dvdy[q] = h22;
    a.exx[q] = e[0];
    a.eyy[q] = e[1];
    a.exy[q] = e[2];
  } else {
    a.dudx[q] = a.dudy[q] = a.dvdx[q] = a.dvdy[q] = nan_;
    a.exx[q] = a.eyy[q] = a.exy[q] = nan_;
  }
  a.valid[q] = ok ? 1 : 0;
}

}  // namespace

cudaError_t launch_strain(const StrainArgs& a, cudaStream_t s) {
  const int h = (a.window - 1) / 2;
  const int SX = kTileX + 2 * h, SY = kTileY + 2 * h;
  const size_t smem = (sizeof(double) + sizeof(float)) * 2 * static_cast<size_t>(SY) * SX +
                      sizeof(float) * 6 * static_cast<size_t>(SY) * kTileX;
  dim3 grid((a.nx + kTileX - 1) / kTileX, (a.ny + kTileY - 1) / kTileY);
  if (h <= kSmallHalf) {
    strain_kernel<staged_per_thread(kSmallHalf)><<<grid, kTileX * kTileY, smem, s>>>(a);
    return cudaGetLastError();
  }
  // the largest window (31) needs about 103 KB; the limit is raised once (thread-safe)
  static const cudaError_t configured = cudaFuncSetAttribute(
      strain_kernel<staged_per_thread(kMaxHalf)>, cudaFuncAttributeMaxDynamicSharedMemorySize, 112 * 1024);
  if (configured != cudaSuccess) return configured;
  strain_kernel<staged_per_thread(kMaxHalf)><<<grid, kTileX * kTileY, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dic
