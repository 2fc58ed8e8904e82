// Integer-pixel seed search: for every seed, the ZNCC between the reference subset
// and the deformed subset shifted by each integer offset (du, dv), |du|, |dv| <= R,
// whose pixels all lie inside the deformed image. Integer gray levels are summed
// exactly in 64-bit integers and normalised once in FP64:
//     C = (N Sfg - Sf Sg) / sqrt((N Sff - Sf^2) (N Sgg - Sg^2)),
// so ranking ties are decided on exact values. The best offset (larger C, then
// smaller |du|+|dv|, then smaller dv, then smaller du) starts the seed's IC-GN
// (Sec. 2.2 leaves the initial estimate to an FFT stage; a brute-force integer
// search gives the same integer start for a seed).
#include <math.h>

#include "dic_internal.cuh"

namespace dic {
namespace {

constexpr double kNoScore = -2.0;    // offset not usable (out of the image or flat)
constexpr double kFlatRef = -3.0;    // the reference subset itself is flat

__device__ __forceinline__ bool integer_gray(int dtype) { return dtype == DIC_U8 || dtype == DIC_U16; }

// grid (2R+1, n_seeds): block y = seed, block x = dv + R; threads stride over du
__global__ void __launch_bounds__(128) seed_scores_kernel(SeedArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int s = blockIdx.y;
  const int dv = static_cast<int>(blockIdx.x) - a.R;
  const int S = a.S, r = (a.S - 1) / 2, N = S * S;
  const int xc = a.seed_xy[2 * s], yc = a.seed_xy[2 * s + 1];
  const int side = 2 * a.R + 1;
  double* out = a.scores + static_cast<int64_t>(s) * side * side + (dv + a.R) * side;
  const bool exact = integer_gray(a.ref.dtype) && integer_gray(a.def.dtype);

  if (exact) {
    int32_t* f = reinterpret_cast<int32_t*>(smem_raw);
    for (int e = threadIdx.x; e < N; e += blockDim.x)
      f[e] = static_cast<int32_t>(load_gray<float>(a.ref, xc - r + e % S, yc - r + e / S));
    __syncthreads();
    int64_t Sf = 0, Sff = 0;
    for (int e = 0; e < N; ++e) {
      Sf += f[e];
      Sff += static_cast<int64_t>(f[e]) * f[e];
    }
    const int64_t Df = static_cast<int64_t>(N) * Sff - Sf * Sf;
    for (int du = threadIdx.x - a.R; du <= a.R; du += blockDim.x) {
      const int x0 = xc + du - r, y0 = yc + dv - r;
      double score = kNoScore;
      if (Df == 0) {
        score = kFlatRef;
      } else if (x0 >= 0 && y0 >= 0 && x0 + S <= a.W && y0 + S <= a.H) {
        int64_t Sg = 0, Sgg = 0, Sfg = 0;
        for (int yy = 0; yy < S; ++yy) {
          for (int xx = 0; xx < S; ++xx) {
            const int64_t g = static_cast<int64_t>(load_gray<float>(a.def, x0 + xx, y0 + yy));
            Sg += g;
            Sgg += g * g;
            Sfg += g * f[yy * S + xx];
          }
        }
        const int64_t Dg = static_cast<int64_t>(N) * Sgg - Sg * Sg;
        if (Dg != 0) {
          const int64_t num = static_cast<int64_t>(N) * Sfg - Sf * Sg;
          score = static_cast<double>(num) /
                  sqrt(static_cast<double>(Df) * static_cast<double>(Dg));
        }
      }
      out[du + a.R] = score;
    }
  } else {
    double* f = reinterpret_cast<double*>(smem_raw);
    for (int e = threadIdx.x; e < N; e += blockDim.x)
      f[e] = load_gray<double>(a.ref, xc - r + e % S, yc - r + e / S);
    __syncthreads();
    double Sf = 0.0, Sff = 0.0;
    for (int e = 0; e < N; ++e) {
      Sf += f[e];
      Sff += f[e] * f[e];
    }
    const double Df = N * Sff - Sf * Sf;
    for (int du = threadIdx.x - a.R; du <= a.R; du += blockDim.x) {
      const int x0 = xc + du - r, y0 = yc + dv - r;
      double score = kNoScore;
      if (!(Df > 0.0)) {
        score = kFlatRef;
      } else if (x0 >= 0 && y0 >= 0 && x0 + S <= a.W && y0 + S <= a.H) {
        double Sg = 0.0, Sgg = 0.0, Sfg = 0.0;
        for (int yy = 0; yy < S; ++yy)
          for (int xx = 0; xx < S; ++xx) {
            const double g = load_gray<double>(a.def, x0 + xx, y0 + yy);
            Sg += g;
            Sgg += g * g;
            Sfg += g * f[yy * S + xx];
          }
        const double Dg = N * Sgg - Sg * Sg;
        if (Dg > 0.0) score = (N * Sfg - Sf * Sg) / sqrt(Df * Dg);
      }
      out[du + a.R] = score;
    }
  }
}

// one block per seed: the best offset (larger C, then smaller |du|+|dv|, then
// smaller dv, then smaller du) into best[s]; -1 if no offset is usable, -2 if the
// reference subset is flat
__global__ void __launch_bounds__(256) seed_best_kernel(SeedCommitArgs a) {
  const int s = blockIdx.x;
  const int side = 2 * a.R + 1;
  const double* sc = a.scores + static_cast<int64_t>(s) * side * side;
  double bc = 0.0;
  int bkey = 0x7fffffff, be = -1, flat = 0;
  for (int e = threadIdx.x; e < side * side; e += blockDim.x) {
    const double c = sc[e];
    if (c == kFlatRef) flat = 1;
    if (c < -1.5) continue;
    const int du = e % side - a.R, dv = e / side - a.R;
    const int key = ((abs(du) + abs(dv)) * (side + 1) + (dv + a.R)) * (side + 1) + (du + a.R);
    if (be < 0 || c > bc || (c == bc && key < bkey)) {
      be = e;
      bc = c;
      bkey = key;
    }
  }
  __shared__ double s_c[8];
  __shared__ int s_k[8], s_e[8], s_f[8];
  for (int o = 16; o > 0; o >>= 1) {
    const double oc = __shfl_xor_sync(0xffffffffu, bc, o);
    const int ok = __shfl_xor_sync(0xffffffffu, bkey, o);
    const int oe = __shfl_xor_sync(0xffffffffu, be, o);
    flat |= __shfl_xor_sync(0xffffffffu, flat, o);
    if (oe >= 0 && (be < 0 || oc > bc || (oc == bc && ok < bkey))) {
      bc = oc;
      bkey = ok;
      be = oe;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_c[warp] = bc;
    s_k[warp] = bkey;
    s_e[warp] = be;
    s_f[warp] = flat;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < static_cast<int>(blockDim.x / 32); ++w) {
      flat |= s_f[w];
      if (s_e[w] >= 0 && (be < 0 || s_c[w] > bc || (s_c[w] == bc && s_k[w] < bkey))) {
        bc = s_c[w];
        bkey = s_k[w];
        be = s_e[w];
      }
    }
    a.best[s] = be >= 0 ? be : (flat ? -2 : -1);
  }
}

// one thread: seeds in the order given, duplicates and out-of-ROI seeds skipped
__global__ void seed_commit_kernel(SeedCommitArgs a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int side = 2 * a.R + 1;
  int count = 0;
  for (int s = 0; s < a.n_seeds; ++s) {
    const int q = a.seed_q[s];
    if (a.roi_ok && !a.roi_ok[q]) continue;
    if (a.wave[q] >= 0) continue;
    a.wave[q] = 0;
    double* p = a.p + static_cast<int64_t>(q) * a.nparams;
    if (a.fft_u) {
      for (int c = 0; c < a.nparams; ++c) p[c] = 0.0;
      p[0] = floor(static_cast<double>(a.fft_u[q]) + 0.5);
      p[1] = floor(static_cast<double>(a.fft_v[q]) + 0.5);
      a.frontier0[count++] = q;
      continue;
    }
    const int best = a.best[s];
    if (best < 0) {
      a.status[q] = best == -2 ? DIC_PT_FLAT : DIC_PT_OUT_OF_BOUNDS;
      continue;
    }
    for (int c = 0; c < a.nparams; ++c) p[c] = 0.0;
    p[0] = static_cast<double>(best % side - a.R);
    p[1] = static_cast<double>(best / side - a.R);
    a.frontier0[count++] = q;
  }
  a.counters[kCount + 0] = count;
  a.counters[kCount + 1] = 0;
  a.counters[kCount + 2] = 0;
  a.counters[kWork + 0] = 0;
  a.counters[kWork + 1] = 0;
  a.counters[kWork + 2] = 0;
}

}  // namespace

cudaError_t launch_seed_scores(const SeedArgs& a, cudaStream_t s) {
  const bool exact = (a.ref.dtype == DIC_U8 || a.ref.dtype == DIC_U16) &&
                     (a.def.dtype == DIC_U8 || a.def.dtype == DIC_U16);
  const size_t smem = static_cast<size_t>(a.S) * a.S * (exact ? sizeof(int32_t) : sizeof(double));
  dim3 grid(2 * a.R + 1, a.n_seeds);
  seed_scores_kernel<<<grid, 128, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_seed_commit(const SeedCommitArgs& a, cudaStream_t s) {
  if (!a.fft_u) seed_best_kernel<<<a.n_seeds, 256, 0, s>>>(a);
  seed_commit_kernel<<<1, 32, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dic
