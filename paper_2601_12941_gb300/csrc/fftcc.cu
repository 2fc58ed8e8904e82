// Multi-window FFT cross-correlation (Sec. 2.2, Eq. 1): rigid displacement
// estimates of square windows, coarse to fine, with the median-absolute-deviation
// outlier removal of Sec. 4 after every level and an optional Gaussian peak fit.
//
// Per window (side L, reference origin (x0, y0), deformed origin (gx0, gy0)):
//   z = (f - f_m) + i (g - g_m) packs both real windows into one complex one, so a
//   single 2-D transform Z gives F(k) = (Z(k) + conj Z(-k)) / 2 and
//   G(k) = (Z(k) - conj Z(-k)) / 2i. The cross power of Eq. 1's numerator is then
//       F conj(G)(k) = Im(Z(k) Z(-k)) / 2 + i (|Z(k)|^2 - |Z(-k)|^2) / 4,
//   whose inverse transform is the circular cross-correlation; divided by
//   ||f - f_m|| ||g - g_m|| it is the zero-normalised correlation R (Eq. 1 with the
//   norms of the transforms in the denominator). The peak of R sits at minus the
//   shift of the deformed window's content.
//
// Three paths:
//   * L <= 32 (the subset-sized last level and the 32 px level): one warp per window,
//     the 2-D DFT as matrix products on the tensor cores (split FP16 operands).
//   * L <= 64 otherwise (the 64 px level, odd sizes 33-63): one block per window, the
//     whole window in shared memory; radix-8 Stockham FFTs (then one radix-4 or
//     radix-2 pass) along rows and columns for powers of two, a direct DFT for odd
//     sizes.
//   * 128 <= L <= 4096: the window in a global work buffer; row FFTs, an in-place
//     tile transpose, paired-row FFTs that form the cross power and transform it
//     back, a transpose back and the inverse row FFTs with a per-window arg-max
//     (packed 64-bit keys: the larger R, ties to the lower row-major index).
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <cuda_fp16.h>

#include <type_traits>

#include "dic_internal.cuh"

namespace dic {
namespace {

constexpr int kSmallThreads = 256;
constexpr int kLineThreads = 512;
constexpr int kLineElems = 4096;       // complex elements per block of the line kernels
constexpr int kTransposeTile = 32;
constexpr int kTrRun = 8;              // rows per column run of the transposed work-buffer I/O

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// The cross power F conj(G) at k from the packed spectrum values Z(k) and Z(-k).
__device__ __forceinline__ float2 cross_power(float2 zk, float2 zm) {
  const float im_prod = zk.x * zm.y + zk.y * zm.x;                  // Im(Z(k) Z(-k))
  const float d = (zk.x * zk.x + zk.y * zk.y) - (zm.x * zm.x + zm.y * zm.y);
  return make_float2(0.5f * im_prod, 0.25f * d);
}

// Orderable key of (value, index): the larger value wins, ties to the lower index.
__device__ __forceinline__ unsigned long long peak_key(float v, int idx) {
  uint32_t u = __float_as_uint(v);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return (static_cast<unsigned long long>(u) << 32) | (0xFFFFFFFFu - static_cast<uint32_t>(idx));
}
__device__ __forceinline__ float key_value(unsigned long long k) {
  uint32_t u = static_cast<uint32_t>(k >> 32);
  u = (u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u;
  return __uint_as_float(u);
}
__device__ __forceinline__ int key_index(unsigned long long k) {
  return static_cast<int>(0xFFFFFFFFu - static_cast<uint32_t>(k & 0xFFFFFFFFu));
}

// A window takes part when both its reference and deformed squares lie inside the
// images (x0 < 0 marks a window to skip); anything else is skipped, never read.
__device__ __forceinline__ bool window_ok(int4 o, int L, int W, int H) {
  return o.x >= 0 && o.y >= 0 && o.z >= 0 && o.w >= 0 && o.x <= W - L && o.y <= H - L && o.z <= W - L &&
         o.w <= H - L;
}

// d = wrap(-k): the shift of the deformed window's content from the peak index k.
__device__ __forceinline__ int shift_of_peak(int k, int L) {
  const int h = L / 2;
  int m = (-k + h) % L;
  if (m < 0) m += L;
  return m - h;
}

// Vertex offset of the Gaussian through three samples (0 unless all are positive
// and the middle one is a strict maximum of the fitted parabola of logarithms).
__device__ __forceinline__ float gauss3(float rm, float r0, float rp) {
  if (!(rm > 0.f && r0 > 0.f && rp > 0.f)) return 0.f;
  const float lm = logf(rm), l0 = logf(r0), lp = logf(rp);
  const float den = 2.f * (lm - 2.f * l0 + lp);
  if (!(den < 0.f)) return 0.f;
  return (lm - lp) / den;
}

// exp(-2 pi i m / M) (conjugated for the inverse), 0 <= m < M, M a power of two
// >= 2, from the nested table tw[ns - 1 + k] = exp(-2 pi i k / (2 ns)), k < ns.
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int m, int M, bool inv) {
  const int h = M >> 1;
  float2 w = m < h ? tw[h - 1 + m] : tw[m - 1];          // m >= h: the entry of m - h, negated
  if (m >= h) {
    w.x = -w.x;
    w.y = -w.y;
  }
  if (inv) w.y = -w.y;
  return w;
}

// Shared-memory slot of element e of a transform buffer: one pad slot after every 8, so
// that the stride-R stores of the first Stockham passes and the strided column
// accesses fall on distinct banks. A buffer of n elements takes fft_slots(n) slots.
__host__ __device__ __forceinline__ int fsl(int e) { return e + (e >> 3); }
__host__ __device__ __forceinline__ int fft_slots(int n) { return n + (n >> 3); }

// DFT of 4 points in place, forward (exp(-2 pi i n k / 4)) or inverse.
template <bool INV>
__device__ __forceinline__ void dft4(float2& y0, float2& y1, float2& y2, float2& y3) {
  const float2 t0 = cadd(y0, y2), t1 = csub(y0, y2), t2 = cadd(y1, y3), t3 = csub(y1, y3);
  const float2 rt = INV ? make_float2(-t3.y, t3.x) : make_float2(t3.y, -t3.x);   // +-i t3
  y0 = cadd(t0, t2);
  y2 = csub(t0, t2);
  y1 = cadd(t1, rt);
  y3 = csub(t1, rt);
}

// DFT of 8 points in place: the 4-point DFTs of the even and odd samples combined
// with exp(-+2 pi i k / 8).
template <bool INV>
__device__ __forceinline__ void dft8(float2 (&v)[8]) {
  constexpr float h = 0.70710678118654752f;             // sqrt(1/2)
  dft4<INV>(v[0], v[2], v[4], v[6]);
  dft4<INV>(v[1], v[3], v[5], v[7]);
  float2 b1 = v[3], b2 = v[5], b3 = v[7];               // odd DFT's outputs 1, 2, 3
  if (INV) {
    b1 = make_float2(h * (b1.x - b1.y), h * (b1.x + b1.y));       // x exp(i pi / 4)
    b2 = make_float2(-b2.y, b2.x);                                // x i
    b3 = make_float2(-h * (b3.x + b3.y), h * (b3.x - b3.y));      // x exp(3 i pi / 4)
  } else {
    b1 = make_float2(h * (b1.x + b1.y), h * (b1.y - b1.x));       // x exp(-i pi / 4)
    b2 = make_float2(b2.y, -b2.x);                                // x -i
    b3 = make_float2(h * (b3.y - b3.x), -h * (b3.x + b3.y));      // x exp(-3 i pi / 4)
  }
  const float2 a0 = v[0], a1 = v[2], a2 = v[4], a3 = v[6], b0 = v[1];
  v[0] = cadd(a0, b0);
  v[4] = csub(a0, b0);
  v[1] = cadd(a1, b1);
  v[5] = csub(a1, b1);
  v[2] = cadd(a2, b2);
  v[6] = csub(a2, b2);
  v[3] = cadd(a3, b3);
  v[7] = csub(a3, b3);
}

template <int R, bool INV>
__device__ __forceinline__ void dft_r(float2 (&v)[R]) {
  if constexpr (R == 8) {
    dft8<INV>(v);
  } else if constexpr (R == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  } else {
    const float2 a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  }
}

// One Stockham pass of radix R after sub-transforms of size ns over `lines` lines of
// length L: butterfly j takes its inputs at j + r L / R, twiddles them by
// exp(-+2 pi i r (j mod ns) / (R ns)) and writes output r at
// (j - j mod ns) R + j mod ns + r ns. Element i of line l sits at slot
// fsl(l * ls + i * es). Along rows (es = 1) consecutive threads take consecutive j;
// along columns, consecutive lines.
template <int R, bool INV>
__device__ __forceinline__ void stockham_pass(const float2* __restrict__ in, float2* __restrict__ out, int L,
                                              int lines, int ls, int es, int ns, const float2* __restrict__ tw) {
  const int nb = L / R, lgb = __ffs(nb) - 1, lgl = __ffs(lines) - 1;
  const int total = lines * nb;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int l, j;
    if (es == 1) {
      l = t >> lgb;
      j = t & (nb - 1);
    } else {
      j = t >> lgl;
      l = t & (lines - 1);
    }
    const int base = l * ls, k = j & (ns - 1);
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[fsl(base + (j + r * nb) * es)];
    if (ns > 1) {
      if constexpr (R == 8) {   // w^1, w^2, w^4 from the table, the other powers as products
        const float2 w1 = twiddle(tw, k, 8 * ns, INV), w2 = twiddle(tw, 2 * k, 8 * ns, INV),
                     w4 = twiddle(tw, 4 * k, 8 * ns, INV);
        const float2 w3 = cmul(w1, w2);
        v[1] = cmul(v[1], w1);
        v[2] = cmul(v[2], w2);
        v[3] = cmul(v[3], w3);
        v[4] = cmul(v[4], w4);
        v[5] = cmul(v[5], cmul(w1, w4));
        v[6] = cmul(v[6], cmul(w2, w4));
        v[7] = cmul(v[7], cmul(w3, w4));
      } else {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twiddle(tw, r * k, R * ns, INV));
      }
    }
    dft_r<R, INV>(v);
    const int d = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) out[fsl(base + (d + r * ns) * es)] = v[r];
  }
  __syncthreads();
}

// Transforms `lines` lines of length L (a power of two >= 2; `lines` a power of two):
// radix-8 Stockham passes, then one radix-4 or radix-2 pass for the rest; ping-pong
// between p and q (fft_slots(...) each, padded slots), the result in the returned buffer.
template <bool INV>
__device__ float2* fft_lines(float2* p, float2* q, int L, int lines, int ls, int es, const float2* __restrict__ tw) {
  int ns = 1;
  for (; ns * 8 <= L; ns *= 8) {
    stockham_pass<8, INV>(p, q, L, lines, ls, es, ns, tw);
    float2* t = p;
    p = q;
    q = t;
  }
  if (ns < L) {
    if (L / ns == 4) {
      stockham_pass<4, INV>(p, q, L, lines, ls, es, ns, tw);
    } else {
      stockham_pass<2, INV>(p, q, L, lines, ls, es, ns, tw);
    }
    float2* t = p;
    p = q;
    q = t;
  }
  return p;
}

// acc += p q (complex)
__device__ __forceinline__ void cmac(float2& acc, float2 p, float2 q) {
  acc.x = fmaf(p.x, q.x, fmaf(-p.y, q.y, acc.x));
  acc.y = fmaf(p.x, q.y, fmaf(p.y, q.x, acc.y));
}

// One pass of the 2-D DFT of odd side L as a complex matrix product with the DFT
// matrix Wm[x][k] = exp(-2 pi i x k / L) (symmetric): along rows OUT = IN Wm, along
// columns OUT = Wm IN; INV uses conj(Wm). Each thread accumulates a kTileR x 2 tile
// of OUT over the L terms: kTileR + 2 complex loads (the kTileR row operands are
// broadcast within a warp) for 2 kTileR complex multiply-adds. Only the first
// rows_out rows of OUT are formed.
constexpr int kTileR = 4;
template <bool ROWS, bool INV>
__device__ void dft_matmul(const float2* __restrict__ in, float2* __restrict__ out, const float2* __restrict__ Wm,
                           int L, int rows_out) {
  const int ntc = (L + 1) >> 1, ntr = (rows_out + kTileR - 1) / kTileR;
  for (int t = threadIdx.x; t < ntr * ntc; t += blockDim.x) {
    const int r0 = (t / ntc) * kTileR, c0 = (t - (t / ntc) * ntc) * 2;
    const int c1 = min(c0 + 1, L - 1);
    int rr[kTileR];
#pragma unroll
    for (int i = 0; i < kTileR; ++i) rr[i] = min(r0 + i, L - 1);
    float2 acc0[kTileR], acc1[kTileR];
#pragma unroll
    for (int i = 0; i < kTileR; ++i) acc0[i] = acc1[i] = make_float2(0.f, 0.f);
    for (int x = 0; x < L; ++x) {
      float2 p[kTileR], q0, q1;
      if (ROWS) {
#pragma unroll
        for (int i = 0; i < kTileR; ++i) p[i] = in[rr[i] * L + x];
        q0 = Wm[x * L + c0];
        q1 = Wm[x * L + c1];
        if (INV) {
          q0.y = -q0.y;
          q1.y = -q1.y;
        }
      } else {
#pragma unroll
        for (int i = 0; i < kTileR; ++i) {
          p[i] = Wm[rr[i] * L + x];
          if (INV) p[i].y = -p[i].y;
        }
        q0 = in[x * L + c0];
        q1 = in[x * L + c1];
      }
#pragma unroll
      for (int i = 0; i < kTileR; ++i) {
        cmac(acc0[i], p[i], q0);
        cmac(acc1[i], p[i], q1);
      }
    }
#pragma unroll
    for (int i = 0; i < kTileR; ++i) {
      if (r0 + i < rows_out) {
        out[(r0 + i) * L + c0] = acc0[i];
        if (c0 + 1 < L) out[(r0 + i) * L + c0 + 1] = acc1[i];
      }
    }
  }
  __syncthreads();
}

// The last inverse pass for a Hermitian spectrum: T holds the inverse row transforms
// of rows ky = 0 .. (L-1)/2 only (the others are their conjugates, T[-ky] = conj T[ky]),
// and R[y][x] = Re T[0][x] + 2 sum_{ky >= 1} Re(T[ky][x] exp(2 pi i ky y / L)), the real
// part only (R is real). kTileR x 2 tiles of R; R is written as the .x of out.
__device__ void dft_inverse_columns_real(const float2* __restrict__ T, float2* __restrict__ out,
                                         const float2* __restrict__ Wm, int L) {
  const int ntc = (L + 1) >> 1, ntr = (L + kTileR - 1) / kTileR, kh = (L + 1) >> 1;
  for (int t = threadIdx.x; t < ntr * ntc; t += blockDim.x) {
    const int r0 = (t / ntc) * kTileR, c0 = (t - (t / ntc) * ntc) * 2;
    const int c1 = min(c0 + 1, L - 1);
    int rr[kTileR];
#pragma unroll
    for (int i = 0; i < kTileR; ++i) rr[i] = min(r0 + i, L - 1);
    float acc0[kTileR], acc1[kTileR];
#pragma unroll
    for (int i = 0; i < kTileR; ++i) {                 // the ky = 0 term, halved
      acc0[i] = 0.5f * T[c0].x;
      acc1[i] = 0.5f * T[c1].x;
    }
    for (int ky = 1; ky < kh; ++ky) {
      const float2 q0 = T[ky * L + c0], q1 = T[ky * L + c1];
#pragma unroll
      for (int i = 0; i < kTileR; ++i) {
        const float2 p = Wm[rr[i] * L + ky];           // exp(-2 pi i ky y / L)
        // Re(q conj(p)) = q.x p.x + q.y p.y
        acc0[i] = fmaf(q0.x, p.x, fmaf(q0.y, p.y, acc0[i]));
        acc1[i] = fmaf(q1.x, p.x, fmaf(q1.y, p.y, acc1[i]));
      }
    }
#pragma unroll
    for (int i = 0; i < kTileR; ++i) {
      if (r0 + i < L) {
        out[(r0 + i) * L + c0].x = 2.f * acc0[i];
        if (c0 + 1 < L) out[(r0 + i) * L + c0 + 1].x = 2.f * acc1[i];
      }
    }
  }
  __syncthreads();
}

template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Sums of two values over the block (all threads get them). FP32: the sums only set
// the windows' means and the normalisation of R, and FP64 arithmetic in every thread
// would bind these kernels on this GPU's FP64 pipe.
__device__ void block_sum2(float& a, float& b, float* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  __syncthreads();
  if (lane == 0) {
    scratch[2 * wid] = a;
    scratch[2 * wid + 1] = b;
  }
  __syncthreads();
  a = 0.f;
  b = 0.f;
  for (int w = 0; w < nw; ++w) {
    a += scratch[2 * w];
    b += scratch[2 * w + 1];
  }
}

__device__ unsigned long long block_max_key(unsigned long long v, unsigned long long* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max_key(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  v = 0ull;
  for (int w = 0; w < nw; ++w) v = scratch[w] > v ? scratch[w] : v;
  return v;
}

// ---------------------------------------------------------------- small windows
// power-of-two windows: 256 threads; odd (the last level): 128, which the kTileR x 2
// tiles of a 31 x 31 window fill exactly
template <bool POW2>
__global__ void __launch_bounds__(POW2 ? kSmallThreads : kSmallThreads / 2) fftcc_small_kernel(FftccArgs a) {
  constexpr int NT = POW2 ? kSmallThreads : kSmallThreads / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = a.L, N = L * L, NS = POW2 ? fft_slots(N) : N;
  float2* A = reinterpret_cast<float2*>(smem_raw);      // element e at slot sl(e): padded for the FFT passes
  float2* B = A + NS;
  float2* tws = B + NS;                                  // L - 1 twiddles (power of two) or the L x L DFT matrix
  auto sl = [](int e) { return POW2 ? fsl(e) : e; };
  const int lg = __ffs(L) - 1;                           // POW2: e / L = e >> lg
  auto row_of = [&](int e) { return POW2 ? e >> lg : e / L; };
  __shared__ float s_red[2 * (kSmallThreads / 32)];
  __shared__ unsigned long long s_key[kSmallThreads / 32];
  const int tid = threadIdx.x;
  // the nested power-of-two table: stage ns <= L/2 reads tw_pow2[ns - 1 + k], k < ns,
  // so the block keeps entries 0 .. L - 2
  if (POW2) {
    for (int e = tid; e < L - 1; e += NT) tws[e] = a.tw_pow2[e];
  } else {
    for (int e = tid; e < N; e += NT) {
      const int x = e / L, k = e - x * L;
      tws[e] = a.tw_odd[(x * k) % L];
    }
  }
  __syncthreads();

  for (int64_t w = blockIdx.x; w < a.n; w += gridDim.x) {
    const int4 o = a.org[w];
    if (!window_ok(o, L, a.W, a.H)) {                    // skipped (outside the ROI)
      if (tid == 0) {
        a.u[w] = 0.f;
        a.v[w] = 0.f;
        a.peak[w] = 0.f;
      }
      continue;
    }
    // FP32 sums (FP64 arithmetic in every thread would bind the kernel on this GPU's
    // FP64 pipe); they set the means and the normalisation of R only
    float pf = 0.f, pg = 0.f;
    const float f00 = load_gray<float>(a.ref, o.x, o.y), g00 = load_gray<float>(a.def, o.z, o.w);
    bool vf = false, vg = false;                         // a value differs from the first
    for (int e = tid; e < N; e += NT) {
      const int y = row_of(e), x = e - y * L;
      const float f = load_gray<float>(a.ref, o.x + x, o.y + y);
      const float g = load_gray<float>(a.def, o.z + x, o.w + y);
      A[sl(e)] = make_float2(f, g);
      pf += f;
      pg += g;
      vf |= f != f00;
      vg |= g != g00;
    }
    float sf = pf, sg = pg;
    const int any_f = __syncthreads_or(vf);
    const int any_g = __syncthreads_or(vg);
    const bool flat = !any_f || !any_g;
    block_sum2(sf, sg, s_red);
    const float mf = sf / static_cast<float>(N), mg = sg / static_cast<float>(N);
    float pqf = 0.f, pqg = 0.f;
    for (int e = tid; e < N; e += NT) {
      float2 v = A[sl(e)];
      v.x -= mf;
      v.y -= mg;
      A[sl(e)] = v;
      pqf = fmaf(v.x, v.x, pqf);
      pqg = fmaf(v.y, v.y, pqg);
    }
    float qf = pqf, qg = pqg;
    block_sum2(qf, qg, s_red);                           // (its barriers also order the writes above)
    float2* X;
    float2* Y;
    if (POW2) {
      X = fft_lines<false>(A, B, L, L, L, 1, tws);       // rows
      Y = X == A ? B : A;
      X = fft_lines<false>(X, Y, L, L, 1, L, tws);       // columns
    } else {
      dft_matmul<true, false>(A, B, tws, L, L);
      dft_matmul<false, false>(B, A, tws, L, L);
      X = A;
    }
    Y = X == A ? B : A;
    for (int e = tid; e < N; e += NT) {
      const int ky = row_of(e), kx = e - ky * L;
      const int m = (ky == 0 ? 0 : L - ky) * L + (kx == 0 ? 0 : L - kx);
      Y[sl(e)] = e == 0 ? make_float2(0.f, 0.f) : cross_power(X[sl(e)], X[sl(m)]);
    }
    __syncthreads();
    float2* R;
    if (POW2) {
      R = fft_lines<true>(Y, X, L, L, L, 1, tws);
      float2* S2 = R == A ? B : A;
      R = fft_lines<true>(R, S2, L, L, 1, L, tws);
    } else {
      dft_matmul<true, true>(Y, X, tws, L, (L + 1) / 2);   // rows ky <= (L-1)/2 of the Hermitian half
      dft_inverse_columns_real(X, Y, tws, L);
      R = Y;
    }
    unsigned long long best = 0ull;
    for (int e = tid; e < N; e += NT) {
      const unsigned long long k = peak_key(R[sl(e)].x, e);
      best = k > best ? k : best;
    }
    best = block_max_key(best, s_key);
    if (tid == 0) {
      const int e = flat ? 0 : key_index(best);
      const int ky = row_of(e), kx = e - ky * L;
      float dx = static_cast<float>(shift_of_peak(kx, L)), dy = static_cast<float>(shift_of_peak(ky, L));
      if (a.subpixel && !flat) {
        const int xm = kx == 0 ? L - 1 : kx - 1, xp = kx == L - 1 ? 0 : kx + 1;
        const int ym = ky == 0 ? L - 1 : ky - 1, yp = ky == L - 1 ? 0 : ky + 1;
        const float r0 = R[sl(e)].x;
        dx -= gauss3(R[sl(ky * L + xm)].x, r0, R[sl(ky * L + xp)].x);
        dy -= gauss3(R[sl(ym * L + kx)].x, r0, R[sl(yp * L + kx)].x);
      }
      a.u[w] = static_cast<float>(o.z - o.x) + dx;
      a.v[w] = static_cast<float>(o.w - o.y) + dy;
      a.peak[w] = flat ? 0.f : R[sl(e)].x / (static_cast<float>(N) * sqrtf(qf) * sqrtf(qg));
    }
    __syncthreads();                                     // the next window reuses the buffers
  }
}

// ---------------------------------------------------------------- windows up to 32 px on the tensor cores
// Windows up to 32 px (the subset-sized last level and the 32 px level): the DFT matrix
// products of a window on the tensor cores, mma.sync m16n8k16 with FP16 operands and
// FP32 accumulators, each operand split into an FP16 high part and an FP16 remainder so
// that hi*hi + hi*lo + lo*hi keeps about FP32 accuracy (22 significant bits). Data
// operands are scaled by powers of two before the split (exact) to stay inside the FP16
// range: the window by 2^E1 from its largest centred value, the row transforms by 2^-7
// (|Y| < 2^20), the cross power by 2^E3 from its largest entry, the inverse row
// transforms by 2^-7; the peak value undoes the product of the scales. The window is
// padded to 32; a complex product is a real product in block form ([[Ar, -Ai], [Ai, Ar]]
// on the left, [[Br, Bi], [-Bi, Br]] on the right). With W the DFT matrix (symmetric) and
// Z the packed window:
//   1. Y^T = W Z^T          rows, forward       (64 x 64) x (64 x 32), stored [Yr^T | Yi^T]
//   2. X^T = Y^T W          columns, forward    (32 x 64) x (64 x 64)
//   3. P = cross power of X(k), X(-k), rows ky <= 15 of the Hermitian half, stored
//      conjugated
//   4. U^T = W conj(P)^T    inverse rows        (64 x 64) x (64 x 16); T = conj(U) = P conj(W),
//                           stored as T^T
//   5. R = A6 [Tr; Ti]      R[y][x] = sum_ky c_ky (Tr cos(2 pi ky y / L) - Ti sin(...)),
//                           c_0 = 1, c_ky = 2, and c_{L/2} = 1 for even L: (32 x 32) x (32 x 32)
// Every product reads its data operand in the layout the stage before wrote (pairs along
// the summed index), so no stage stores transposed. For L = 32 the Hermitian half has a
// 17th row, the Nyquist row ky = 16, whose inverse row transform T16 is real: it is
// formed with shuffles (FP32 FMA) and adds T16[x] (-1)^y to R.
// One warp per window, with its own 32 x kH16SA buffer of FP32 values in shared memory,
// so a window needs no block-wide barrier: 16 warps per block (one block per SM, 128
// registers a thread); W and A6 are held once per block as split fragments in fragment
// order (one 16-byte shared load per lane gives a B fragment's high and low parts).
constexpr int kTcP = 32;                  // padded window side
constexpr int kTcSW = kTcP + 8;           // row stride of T^T and of R
constexpr int kTcWarps = 16;
constexpr int kTcBlockThreads = 32 * kTcWarps;
constexpr int kH16SA = 2 * kTcP + 8;      // row stride (floats) of the 32 x 64 data buffers
constexpr int kH16Buf = kTcP * kH16SA;    // floats per warp
constexpr int kWaFrags = 4 * 4 * 2 * 32;  // A fragments of [[Wr, -Wi], [Wi, Wr]]: row tiles x k-steps x (hi, lo) x lanes
constexpr int kWbFrags = 4 * 8 * 32;      // B fragments of [[Wr, Wi], [-Wi, Wr]]: k-steps x column tiles x lanes
constexpr int kA6hFrags = 2 * 2 * 2 * 32; // A fragments of A6: row tiles x k-steps x (hi, lo) x lanes

// Gray levels of a column of the window: rows y < L of pixel column x (lanes x >= L
// and rows y >= L give 0), the element type fixed once per window.
struct Bf16Bits {   // a bfloat16 gray level: the high half of a float
  uint16_t bits;
};

template <typename G>
__device__ __forceinline__ float gray_at(const char* p) {
  if constexpr (sizeof(G) == 1) {
    return static_cast<float>(*reinterpret_cast<const uint8_t*>(p));
  } else if constexpr (std::is_same<G, Bf16Bits>::value) {
    return __uint_as_float(static_cast<uint32_t>(*reinterpret_cast<const uint16_t*>(p)) << 16);
  } else {
    return static_cast<float>(*reinterpret_cast<const G*>(p));
  }
}

// Column `lane` of the window at (x0, y0) into col[y * ld] (zero padded to 32 rows),
// returning the column sum; *varies: a pixel differs from v00.
template <typename G>
__device__ __forceinline__ float window_column(const GrayPlane& pl, int x0, int y0, int L, int lane, float* col,
                                               int ld, float v00, bool* varies) {
  const bool in = lane < L;
  const char* p = static_cast<const char*>(pl.data) + static_cast<int64_t>(y0) * pl.stride +
                  static_cast<int64_t>(x0 + (in ? lane : 0)) * sizeof(G);
  float s = 0.f;
  bool vary = false;
#pragma unroll
  for (int y = 0; y < kTcP; ++y) {
    float v = 0.f;
    if (in && y < L) {
      v = gray_at<G>(p + static_cast<int64_t>(y) * pl.stride);
      vary |= v != v00;
    }
    col[y * ld] = v;
    s += v;
  }
  *varies = vary;
  return s;
}

__device__ __forceinline__ float load_window_column(const GrayPlane& pl, int x0, int y0, int L, int lane, float* col,
                                                    int ld, float v00, bool* varies) {
  switch (pl.dtype) {
    case DIC_U8:
      return window_column<uint8_t>(pl, x0, y0, L, lane, col, ld, v00, varies);
    case DIC_U16:
      return window_column<uint16_t>(pl, x0, y0, L, lane, col, ld, v00, varies);
    case DIC_BF16:
      return window_column<Bf16Bits>(pl, x0, y0, L, lane, col, ld, v00, varies);
    case DIC_F32:
      return window_column<float>(pl, x0, y0, L, lane, col, ld, v00, varies);
    default:
      return window_column<double>(pl, x0, y0, L, lane, col, ld, v00, varies);
  }
}

// c += a b, m16n8k16, FP16 operands (f16x2 registers), FP32 accumulators
__device__ __forceinline__ void mma_f16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// (x0 s, x1 s) as an f16x2 high part and an f16x2 remainder (x0 in the low half)
__device__ __forceinline__ void split_h2(float x0, float x1, float s, uint32_t& hi, uint32_t& lo) {
  const float y0 = x0 * s, y1 = x1 * s;
  const __half2 h = __floats2half2_rn(y0, y1);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(y0 - hf.x, y1 - hf.y);
  memcpy(&hi, &h, sizeof(hi));
  memcpy(&lo, &l, sizeof(lo));
}

// The exponent E = 13 - floor(log2 m), clamped to [-100, 100] (0 for m = 0): m 2^E lies
// in [2^13, 2^14)
__device__ __forceinline__ int f16_scale_exp(float m) {
  if (!(m > 0.f)) return 0;
  const int e = static_cast<int>((__float_as_uint(m) >> 23) & 0xffu) - 127;
  const int E = 13 - e;
  return E < -100 ? -100 : (E > 100 ? 100 : E);
}
// 2^E as a float, -126 <= E <= 127
__device__ __forceinline__ float pow2f(int E) { return __uint_as_float(static_cast<uint32_t>(127 + E) << 23); }

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// A fragments (row tile mt, k-step ks) of an M x K row-major operand given by el(r, c),
// split: lane (g, t) holds rows g, g + 8 and columns 2t, 2t + 1, 2t + 8, 2t + 9.
template <typename F>
__device__ __forceinline__ void a16_fragment(F el, int mt, int ks, int ln, uint4& hi, uint4& lo) {
  const int g = ln >> 2, t = ln & 3, r0 = 16 * mt + g, c0 = 16 * ks + 2 * t;
  uint32_t h[4], l[4];
  split_h2(el(r0, c0), el(r0, c0 + 1), 1.f, h[0], l[0]);
  split_h2(el(r0 + 8, c0), el(r0 + 8, c0 + 1), 1.f, h[1], l[1]);
  split_h2(el(r0, c0 + 8), el(r0, c0 + 9), 1.f, h[2], l[2]);
  split_h2(el(r0 + 8, c0 + 8), el(r0 + 8, c0 + 9), 1.f, h[3], l[3]);
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// The DFT matrix W[x][k] = exp(-2 pi i x k / L) (x, k < L; else 0) from the root table
__device__ __forceinline__ float2 w_entry(const float2* __restrict__ tw, int L, int x, int k) {
  return (x < L && k < L) ? tw[(x * k) % L] : make_float2(0.f, 0.f);
}

__global__ void __launch_bounds__(kTcBlockThreads, 1) fftcc_tc_kernel(FftccArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float2 s_root[kTcP];                           // exp(-2 pi i m / L), m < L
  const int L = a.L, N = L * L, kh = L / 2 + 1;             // rows 0 .. L/2 of the Hermitian half
  const bool nyquist = L == 32;                             // row ky = 16, outside the 16-row tile
  uint4* wa = reinterpret_cast<uint4*>(smem_raw);          // A fragments of [[Wr, -Wi], [Wi, Wr]]
  uint4* wb = wa + kWaFrags;                                // B fragments of [[Wr, Wi], [-Wi, Wr]]
  uint4* a6f = wb + kWbFrags;                               // A fragments of A6
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* buf = reinterpret_cast<float*>(a6f + kA6hFrags) + warp * kH16Buf;
  const int g = lane >> 2, t = lane & 3;

  const bool pow2 = (L & (L - 1)) == 0;
  for (int e = tid; e < L; e += kTcBlockThreads) s_root[e] = pow2 ? twiddle(a.tw_pow2, e, L, false) : a.tw_odd[e];
  __syncthreads();
  // [[Wr, -Wi], [Wi, Wr]] as A fragments: entry ((mt, ks), hi/lo, lane)
  for (int e = tid; e < kWaFrags / 2; e += kTcBlockThreads) {
    const int mt = e >> 7, ks = (e >> 5) & 3, ln = e & 31;
    uint4 hi, lo;
    a16_fragment([&](int r, int c) {
      const float2 w = w_entry(s_root, L, r & 31, c & 31);
      const int qr = r >> 5, qc = c >> 5;
      return qr == qc ? w.x : (qr == 0 ? -w.y : w.y);
    }, mt, ks, ln, hi, lo);
    wa[2 * e - ln] = hi;
    wa[2 * e - ln + 32] = lo;
  }
  // [[Wr, Wi], [-Wi, Wr]] as B fragments: entry (ks, nt, lane) = (hi b01, hi b23, lo b01, lo b23);
  // lane (g, t) holds rows 2t, 2t + 1, 2t + 8, 2t + 9 of column g
  for (int e = tid; e < kWbFrags; e += kTcBlockThreads) {
    const int ks = e >> 8, nt = (e >> 5) & 7, ln = e & 31;
    const int n = 8 * nt + (ln >> 2), k0 = 16 * ks + 2 * (ln & 3);
    auto el = [&](int r, int c) {
      const float2 w = w_entry(s_root, L, r & 31, c & 31);
      const int qr = r >> 5, qc = c >> 5;
      return qr == qc ? w.x : (qr == 0 ? w.y : -w.y);
    };
    uint32_t h0, l0, h1, l1;
    split_h2(el(k0, n), el(k0 + 1, n), 1.f, h0, l0);
    split_h2(el(k0 + 8, n), el(k0 + 9, n), 1.f, h1, l1);
    wb[e] = make_uint4(h0, h1, l0, l1);
  }
  // A6[y][kp] (y < L): kp < 16 the cosine column of ky = kp, else the sine column of
  // kp - 16, weighted c_0 = 1, c_ky = 2, c_{L/2} = 1 (ky <= L / 2; else 0)
  for (int e = tid; e < kA6hFrags / 2; e += kTcBlockThreads) {
    const int mt = e >> 6, ks = (e >> 5) & 1, ln = e & 31;
    uint4 hi, lo;
    a16_fragment([&](int y, int kp) {
      const int ky = kp & 15;
      if (!(y < L && ky < kh)) return 0.f;
      const float2 q = s_root[(ky * y) % L];              // (cos, -sin) of 2 pi ky y / L
      const float c = (ky == 0 || 2 * ky == L) ? 1.f : 2.f;
      return kp < 16 ? c * q.x : c * q.y;
    }, mt, ks, ln, hi, lo);
    a6f[2 * e - ln] = hi;
    a6f[2 * e - ln + 32] = lo;
  }
  __syncthreads();

  const int64_t stride = static_cast<int64_t>(gridDim.x) * kTcWarps;
  for (int64_t win = static_cast<int64_t>(blockIdx.x) * kTcWarps + warp; win < a.n; win += stride) {
    const int4 o = a.org[win];
    if (!window_ok(o, L, a.W, a.H)) {                       // skipped (outside the ROI)
      if (lane == 0) {
        a.u[win] = 0.f;
        a.v[win] = 0.f;
        a.peak[win] = 0.f;
      }
      continue;
    }
    // the packed window Z = [f | g] in buf (rows y, columns x and 32 + x; zero
    // padding), lane x loading pixel column x; then centred by the means
    const float f00 = load_gray<float>(a.ref, o.x, o.y), g00 = load_gray<float>(a.def, o.z, o.w);
    bool vf, vg;
    float sf = load_window_column(a.ref, o.x, o.y, L, lane, buf + lane, kH16SA, f00, &vf);
    float sg = load_window_column(a.def, o.z, o.w, L, lane, buf + kTcP + lane, kH16SA, g00, &vg);
    const bool flat = !__any_sync(0xffffffffu, vf) || !__any_sync(0xffffffffu, vg);
    sf = warp_sum(sf);
    sg = warp_sum(sg);
    const float mf = sf / static_cast<float>(N), mg = sg / static_cast<float>(N);
    float qf = 0.f, qg = 0.f, zmax = 0.f;
    if (lane < L) {
      for (int y = 0; y < L; ++y) {
        const float f = buf[y * kH16SA + lane] - mf, gv = buf[y * kH16SA + kTcP + lane] - mg;
        buf[y * kH16SA + lane] = f;
        buf[y * kH16SA + kTcP + lane] = gv;
        qf = fmaf(f, f, qf);
        qg = fmaf(gv, gv, qg);
        zmax = fmaxf(zmax, fmaxf(fabsf(f), fabsf(gv)));
      }
    }
    qf = warp_sum(qf);
    qg = warp_sum(qg);
    const int E1 = f16_scale_exp(warp_max(zmax));
    const float s1 = pow2f(E1);
    __syncwarp();

    // 1. Y^T = W Z^T: [Yr^T; Yi^T] = [[Wr, -Wi], [Wi, Wr]] [Zr^T; Zi^T] (64 x 64 by 64 x 32);
    //    stored as [Yr^T | Yi^T] ([kx][y | 32 + y])
    {
      float acc[4][4][4] = {};
#pragma unroll 1
      for (int ks = 0; ks < 4; ++ks) {
        uint32_t bh[4][2], bl[4][2];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const float* p = buf + (8 * nt + g) * kH16SA + 16 * ks + 2 * t;   // Z row y = 8 nt + g
          const float2 v0 = *reinterpret_cast<const float2*>(p), v1 = *reinterpret_cast<const float2*>(p + 8);
          split_h2(v0.x, v0.y, s1, bh[nt][0], bl[nt][0]);
          split_h2(v1.x, v1.y, s1, bh[nt][1], bl[nt][1]);
        }
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
          const uint4 h = wa[((mt * 4 + ks) * 2) * 32 + lane], l = wa[((mt * 4 + ks) * 2 + 1) * 32 + lane];
          const uint32_t ah[4] = {h.x, h.y, h.z, h.w}, al[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) mma_f16(acc[mt][nt], ah, bh[nt][0], bh[nt][1]);
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) mma_f16(acc[mt][nt], ah, bl[nt][0], bl[nt][1]);
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) mma_f16(acc[mt][nt], al, bh[nt][0], bh[nt][1]);
        }
      }
      __syncwarp();
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
          for (int hr = 0; hr < 2; ++hr) {
            const int m = 16 * mt + g + 8 * hr, n = 8 * nt + 2 * t;
            *reinterpret_cast<float2*>(buf + (m & 31) * kH16SA + (m >> 5) * kTcP + n) =
                make_float2(acc[mt][nt][2 * hr], acc[mt][nt][2 * hr + 1]);
          }
      __syncwarp();
    }
    // 2. X^T = Y^T W: [Xr^T | Xi^T] = [Yr^T | Yi^T] [[Wr, Wi], [-Wi, Wr]] ([kx][ky | 32 + ky]);
    //    Y^T enters scaled by 2^-7 (|Y| < 2^20)
    {
      float acc[2][8][4] = {};
      const float s2 = pow2f(-7);
#pragma unroll 1
      for (int ks = 0; ks < 4; ++ks) {
        uint32_t ah[2][4], al[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          const float* p = buf + (16 * mt + g) * kH16SA + 16 * ks + 2 * t;
          const float2 v0 = *reinterpret_cast<const float2*>(p), v1 = *reinterpret_cast<const float2*>(p + 8 * kH16SA);
          const float2 v2 = *reinterpret_cast<const float2*>(p + 8),
                       v3 = *reinterpret_cast<const float2*>(p + 8 * kH16SA + 8);
          split_h2(v0.x, v0.y, s2, ah[mt][0], al[mt][0]);
          split_h2(v1.x, v1.y, s2, ah[mt][1], al[mt][1]);
          split_h2(v2.x, v2.y, s2, ah[mt][2], al[mt][2]);
          split_h2(v3.x, v3.y, s2, ah[mt][3], al[mt][3]);
        }
#pragma unroll
        for (int nt = 0; nt < 8; nt += 2) {
          const uint4 b[2] = {wb[(ks * 8 + nt) * 32 + lane], wb[(ks * 8 + nt + 1) * 32 + lane]};
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) mma_f16(acc[mt][nt + h], ah[mt], b[h].x, b[h].y);
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) mma_f16(acc[mt][nt + h], ah[mt], b[h].z, b[h].w);
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) mma_f16(acc[mt][nt + h], al[mt], b[h].x, b[h].y);
        }
      }
      __syncwarp();
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
          for (int hr = 0; hr < 2; ++hr) {
            const int m = 16 * mt + g + 8 * hr, n = 8 * nt + 2 * t;
            *reinterpret_cast<float2*>(buf + m * kH16SA + n) = make_float2(acc[mt][nt][2 * hr], acc[mt][nt][2 * hr + 1]);
          }
      __syncwarp();
    }
    // 3. the cross power P(ky, kx) of rows ky < 16, stored conjugated ([ky][kx | 32 + kx]);
    //    the zero frequency and the padding are zero. All of X is read before P is written.
    float t16 = 0.f, pmax = 0.f;
    {
      const int ky = lane & 15;
      float2 p[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int kx = 2 * j + (lane >> 4);
        p[j] = make_float2(0.f, 0.f);
        if (ky < kh && kx < L && (ky | kx) != 0) {
          const int mkx = kx == 0 ? 0 : L - kx, mky = ky == 0 ? 0 : L - ky;
          const float2 zk = make_float2(buf[kx * kH16SA + ky], buf[kx * kH16SA + kTcP + ky]);
          const float2 zm = make_float2(buf[mkx * kH16SA + mky], buf[mkx * kH16SA + kTcP + mky]);
          p[j] = cross_power(zk, zm);
          pmax = fmaxf(pmax, fmaxf(fabsf(p[j].x), fabsf(p[j].y)));
        }
      }
      float2 p16 = make_float2(0.f, 0.f);                // the Nyquist row's P(16, kx), kx = lane
      if (nyquist) {
        const int mkx = lane == 0 ? 0 : L - lane;
        p16 = cross_power(make_float2(buf[lane * kH16SA + 16], buf[lane * kH16SA + kTcP + 16]),
                          make_float2(buf[mkx * kH16SA + 16], buf[mkx * kH16SA + kTcP + 16]));
      }
      __syncwarp();
      if (nyquist) {                                     // T16[x] = Re sum_kx P(16, kx) exp(2 pi i kx x / L), x = lane
#pragma unroll 8
        for (int kx = 0; kx < 32; ++kx) {
          const float pr = __shfl_sync(0xffffffffu, p16.x, kx), pi = __shfl_sync(0xffffffffu, p16.y, kx);
          const float2 w = s_root[(lane * kx) & 31];
          t16 = fmaf(pr, w.x, fmaf(pi, w.y, t16));
        }
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int kx = 2 * j + (lane >> 4);
        buf[ky * kH16SA + kx] = p[j].x;
        buf[ky * kH16SA + kTcP + kx] = -p[j].y;          // conj(P)
      }
      __syncwarp();
    }
    const int E3 = f16_scale_exp(warp_max(pmax));
    // 4. U^T = W conj(P)^T: [Ur^T; Ui^T] = [[Wr, -Wi], [Wi, Wr]] [Pr^T; -Pi^T] (64 x 64 by
    //    64 x 16), conj(P) entering scaled by 2^E3; T = conj(U) is stored as T^T
    //    ([x][ky | 16 + ky], row stride kTcSW)
    {
      float acc[4][2][4] = {};
      const float s3 = pow2f(E3);
#pragma unroll 1
      for (int ks = 0; ks < 4; ++ks) {
        uint32_t bh[2][2], bl[2][2];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const float* p = buf + (8 * nt + g) * kH16SA + 16 * ks + 2 * t;   // conj(P) row ky = 8 nt + g
          const float2 v0 = *reinterpret_cast<const float2*>(p), v1 = *reinterpret_cast<const float2*>(p + 8);
          split_h2(v0.x, v0.y, s3, bh[nt][0], bl[nt][0]);
          split_h2(v1.x, v1.y, s3, bh[nt][1], bl[nt][1]);
        }
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
          const uint4 h = wa[((mt * 4 + ks) * 2) * 32 + lane], l = wa[((mt * 4 + ks) * 2 + 1) * 32 + lane];
          const uint32_t ah[4] = {h.x, h.y, h.z, h.w}, al[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) mma_f16(acc[mt][nt], ah, bh[nt][0], bh[nt][1]);
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) mma_f16(acc[mt][nt], ah, bl[nt][0], bl[nt][1]);
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) mma_f16(acc[mt][nt], al, bh[nt][0], bh[nt][1]);
        }
      }
      __syncwarp();
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int hr = 0; hr < 2; ++hr) {
            const int m = 16 * mt + g + 8 * hr, n = 8 * nt + 2 * t;
            const float sg2 = m < 32 ? 1.f : -1.f;     // Ti = -Ui
            *reinterpret_cast<float2*>(buf + (m & 31) * kTcSW + (m >> 5) * 16 + n) =
                make_float2(sg2 * acc[mt][nt][2 * hr], sg2 * acc[mt][nt][2 * hr + 1]);
          }
      __syncwarp();
    }
    // 5. R = A6 [Tr; Ti] (32 x 32 by 32 x 32), [Tr; Ti] entering scaled by 2^-7; then the
    //    arg-max over the L x L values (ties to the lower row-major index y L + x)
    //    straight from the accumulators
    float acc[2][4][4] = {};
    {
      const float s4 = pow2f(-7);
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        uint32_t bh[4][2], bl[4][2];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const float* p = buf + (8 * nt + g) * kTcSW + 16 * ks + 2 * t;   // T^T row x = 8 nt + g
          const float2 v0 = *reinterpret_cast<const float2*>(p), v1 = *reinterpret_cast<const float2*>(p + 8);
          split_h2(v0.x, v0.y, s4, bh[nt][0], bl[nt][0]);
          split_h2(v1.x, v1.y, s4, bh[nt][1], bl[nt][1]);
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          const uint4 h = a6f[((mt * 2 + ks) * 2) * 32 + lane], l = a6f[((mt * 2 + ks) * 2 + 1) * 32 + lane];
          const uint32_t ah[4] = {h.x, h.y, h.z, h.w}, al[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) mma_f16(acc[mt][nt], ah, bh[nt][0], bh[nt][1]);
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) mma_f16(acc[mt][nt], ah, bl[nt][0], bl[nt][1]);
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) mma_f16(acc[mt][nt], al, bh[nt][0], bh[nt][1]);
        }
      }
    }
    if (nyquist) {                                       // R[y][x] += T16[x] (-1)^y, in R's scale
      const float sn = pow2f(E3 - 7);
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const float tv = sn * __shfl_sync(0xffffffffu, t16, 8 * j + 2 * t + c);
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            acc[mt][j][c] += (g & 1) ? -tv : tv;         // row 16 mt + g
            acc[mt][j][2 + c] += (g & 1) ? -tv : tv;     // row 16 mt + g + 8
          }
        }
    }
    unsigned long long best = 0ull;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int y = 16 * mt + g + (i >> 1) * 8, x = 8 * j + 2 * t + (i & 1);
          if (y < L && x < L) {
            const unsigned long long k = peak_key(acc[mt][j][i], y * L + x);
            best = k > best ? k : best;
          }
        }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long o2 = __shfl_xor_sync(0xffffffffu, best, off);
      best = o2 > best ? o2 : best;
    }
    __syncwarp();                                        // T^T is no longer read
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int y = 16 * mt + g + (i >> 1) * 8, x = 8 * j + 2 * t + (i & 1);
          buf[y * kTcSW + x] = acc[mt][j][i];
        }
    __syncwarp();
    if (lane == 0) {
      const int e = flat ? 0 : key_index(best);
      const int ky = e / L, kx = e - ky * L;
      float dx = static_cast<float>(shift_of_peak(kx, L)), dy = static_cast<float>(shift_of_peak(ky, L));
      const float r0 = buf[ky * kTcSW + kx];
      if (a.subpixel && !flat) {
        const int xm = kx == 0 ? L - 1 : kx - 1, xp = kx == L - 1 ? 0 : kx + 1;
        const int ym = ky == 0 ? L - 1 : ky - 1, yp = ky == L - 1 ? 0 : ky + 1;
        dx -= gauss3(buf[ky * kTcSW + xm], r0, buf[ky * kTcSW + xp]);
        dy -= gauss3(buf[ym * kTcSW + kx], r0, buf[yp * kTcSW + kx]);
      }
      a.u[win] = static_cast<float>(o.z - o.x) + dx;
      a.v[win] = static_cast<float>(o.w - o.y) + dy;
      // R here is the correlation times 2^(2 E1 - 7 - 7 + E3 - 7): X carries s1 2^-7, P its
      // square, T the factor 2^E3 and the 2^-7 of step 5
      a.peak[win] = flat ? 0.f : ldexpf(r0, 21 - 2 * E1 - E3) / (static_cast<float>(N) * sqrtf(qf) * sqrtf(qg));
    }
    __syncwarp();                                        // the next window reuses the buffer
  }
}

size_t tc_smem() {
  return sizeof(uint4) * (kWaFrags + kWbFrags + kA6hFrags) + sizeof(float) * kTcWarps * kH16Buf;
}

// ---------------------------------------------------------------- large windows
// Gray levels of elements e = threadIdx.x + i kLineThreads of the block's rows of a
// window (row e / L, column e mod L from (x0, y0)), all loads issued before use.
template <typename G>
__device__ __forceinline__ void line_grays_t(const GrayPlane& pl, int x0, int y0, int L,
                                             float (&v)[kLineElems / kLineThreads]) {
  const char* base = static_cast<const char*>(pl.data) + static_cast<int64_t>(y0) * pl.stride +
                     static_cast<int64_t>(x0) * sizeof(G);
  const int lg = __ffs(L) - 1;
#pragma unroll
  for (int i = 0; i < kLineElems / kLineThreads; ++i) {
    const int e = threadIdx.x + i * kLineThreads;
    v[i] = gray_at<G>(base + static_cast<int64_t>(e >> lg) * pl.stride + static_cast<int64_t>(e & (L - 1)) * sizeof(G));
  }
}

__device__ __forceinline__ void line_grays(const GrayPlane& pl, int x0, int y0, int L,
                                           float (&v)[kLineElems / kLineThreads]) {
  switch (pl.dtype) {
    case DIC_U8:
      line_grays_t<uint8_t>(pl, x0, y0, L, v);
      break;
    case DIC_U16:
      line_grays_t<uint16_t>(pl, x0, y0, L, v);
      break;
    case DIC_BF16:
      line_grays_t<Bf16Bits>(pl, x0, y0, L, v);
      break;
    case DIC_F32:
      line_grays_t<float>(pl, x0, y0, L, v);
      break;
    default:
      line_grays_t<double>(pl, x0, y0, L, v);
  }
}

// Rows of the packed windows, transformed along x: work[w][y][kx]. Also marks the
// windows whose f or g is not constant (an exactly flat window correlates to 0).
// TR: the output goes to the work buffer transposed (work[w][kx][y]), in runs of
// kTrRun rows (64 bytes) per column, so no transpose kernel is needed (L <= 512: at
// least kTrRun rows per block).
template <bool TR>
__global__ void __launch_bounds__(kLineThreads, 3) fftcc_rows_fwd_kernel(FftccArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = a.L;
  const int rows = kLineElems / L;                       // L >= 128: 1 .. 32 rows per block
  float2* P = reinterpret_cast<float2*>(smem_raw);      // element e at slot fsl(e)
  float2* Q = P + fft_slots(kLineElems);
  const int64_t w = blockIdx.x;
  const int4 o = a.org[w];
  if (!window_ok(o, L, a.W, a.H)) return;                // uniform: the whole block
  const int y0 = blockIdx.y * rows;
  const float f00 = load_gray<float>(a.ref, o.x, o.y);
  const float g00 = load_gray<float>(a.def, o.z, o.w);
  bool vf = false, vg = false;
  float fv[kLineElems / kLineThreads], gv[kLineElems / kLineThreads];
  line_grays(a.ref, o.x, o.y + y0, L, fv);
  line_grays(a.def, o.z, o.w + y0, L, gv);
#pragma unroll
  for (int i = 0; i < kLineElems / kLineThreads; ++i) {
    vf |= fv[i] != f00;
    vg |= gv[i] != g00;
    P[fsl(threadIdx.x + i * kLineThreads)] = make_float2(fv[i], gv[i]);
  }
  if (__syncthreads_or(vf) && threadIdx.x == 0) atomicOr(&a.nonflat[2 * w], 1);
  if (__syncthreads_or(vg) && threadIdx.x == 0) atomicOr(&a.nonflat[2 * w + 1], 1);
  const float2* R = fft_lines<false>(P, Q, L, rows, L, 1, a.tw_pow2);
  if (TR) {
    const int lg = __ffs(L) - 1;
    float2* base = a.work + w * static_cast<int64_t>(L) * L + y0;
    for (int it = threadIdx.x; it < (rows / kTrRun) * L; it += kLineThreads) {
      const int kx = it & (L - 1), r = kTrRun * (it >> lg);
      float4* d = reinterpret_cast<float4*>(base + static_cast<int64_t>(kx) * L + r);
#pragma unroll
      for (int i = 0; i < kTrRun / 2; ++i) {
        const float2 v0 = R[fsl((r + 2 * i) * L + kx)], v1 = R[fsl((r + 2 * i + 1) * L + kx)];
        d[i] = make_float4(v0.x, v0.y, v1.x, v1.y);
      }
    }
  } else {
    float2* dst = a.work + w * static_cast<int64_t>(L) * L + static_cast<int64_t>(y0) * L;
    for (int e = threadIdx.x; e < rows * L; e += kLineThreads) dst[e] = R[fsl(e)];
  }
}

// In-place transpose of every L x L window: the block of tile (ti, tj), ti <= tj,
// swaps it with its mirror tile (tj, ti).
__global__ void __launch_bounds__(kTransposeTile * 8) fftcc_transpose_kernel(FftccArgs a) {
  __shared__ float2 t0[kTransposeTile][kTransposeTile + 1];
  __shared__ float2 t1[kTransposeTile][kTransposeTile + 1];
  const int L = a.L, T = L / kTransposeTile;
  const int ti = blockIdx.y % T, tj = blockIdx.y / T;
  if (ti > tj) return;
  const int64_t w = blockIdx.x;
  if (!window_ok(a.org[w], L, a.W, a.H)) return;
  float2* base = a.work + w * static_cast<int64_t>(L) * L;
  const int tx = threadIdx.x & (kTransposeTile - 1), ty = threadIdx.x / kTransposeTile;   // 32 x 8
  for (int r = ty; r < kTransposeTile; r += 8) {
    t0[r][tx] = base[static_cast<int64_t>(ti * kTransposeTile + r) * L + tj * kTransposeTile + tx];
    t1[r][tx] = base[static_cast<int64_t>(tj * kTransposeTile + r) * L + ti * kTransposeTile + tx];
  }
  __syncthreads();
  for (int r = ty; r < kTransposeTile; r += 8) {
    base[static_cast<int64_t>(tj * kTransposeTile + r) * L + ti * kTransposeTile + tx] = t0[tx][r];
    base[static_cast<int64_t>(ti * kTransposeTile + r) * L + tj * kTransposeTile + tx] = t1[tx][r];
  }
}

// After the transpose, row kx holds Z1(y, kx) along y. A unit is the row pair
// (u, L - u) (rows 0 and L/2 pair with themselves): FFT both along y, form the cross
// power of each frequency with its mirror, accumulate the norms of F and G (zero
// frequency excluded), transform back along y, write both rows back.
__global__ void __launch_bounds__(kLineThreads, 3) fftcc_pairs_kernel(FftccArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = a.L;
  const int units = L <= kLineElems / 2 ? kLineElems / 2 / L : 1;   // 2 lines each: 4096 elements (8192 at L = 4096)
  const int lines = 2 * units, lg = __ffs(L) - 1;
  float2* P = reinterpret_cast<float2*>(smem_raw);      // element e at slot fsl(e)
  float2* Q = P + fft_slots(lines * L);
  __shared__ float s_red[2 * (kLineThreads / 32)];
  const int64_t w = blockIdx.x;
  if (!window_ok(a.org[w], L, a.W, a.H)) return;
  const int u0 = blockIdx.y * units;
  const int nunits = L / 2 + 1;
  float2* base = a.work + w * static_cast<int64_t>(L) * L;
  for (int e = threadIdx.x; e < lines * L; e += kLineThreads) {
    const int line = e >> lg, y = e & (L - 1);
    const int u = u0 + (line >> 1);
    float2 v = make_float2(0.f, 0.f);
    if (u < nunits) {
      const int row = (line & 1) ? (L - u) & (L - 1) : u;
      v = base[static_cast<int64_t>(row) * L + y];
    }
    P[fsl(e)] = v;
  }
  __syncthreads();
  float2* X = fft_lines<false>(P, Q, L, lines, L, 1, a.tw_pow2);
  float2* Y = X == P ? Q : P;
  float pnf = 0.f, png = 0.f;                             // FP32 per block, FP64 across blocks
  for (int e = threadIdx.x; e < lines * L; e += kLineThreads) {
    const int line = e >> lg, ky = e & (L - 1);
    const int u = u0 + (line >> 1);
    const int mline = line ^ 1;                          // the mirror row's line
    const int mky = ky == 0 ? 0 : L - ky;
    const float2 zk = X[fsl(e)], zm = X[fsl(mline * L + mky)];
    const bool dc = u == 0 && ky == 0;
    Y[fsl(e)] = dc ? make_float2(0.f, 0.f) : cross_power(zk, zm);
    // each frequency once: line 0 of the unit, and line 1 only when its row differs
    const bool count = u < nunits && !dc && ((line & 1) == 0 || (u != 0 && 2 * u != L));
    if (count) {
      const float fx = 0.5f * (zk.x + zm.x), fy = 0.5f * (zk.y - zm.y);   // F(k)
      const float gx = 0.5f * (zk.y + zm.y), gy = 0.5f * (zm.x - zk.x);   // G(k)
      pnf = fmaf(fx, fx, fmaf(fy, fy, pnf));
      png = fmaf(gx, gx, fmaf(gy, gy, png));
    }
  }
  float nf = pnf, ng = png;
  block_sum2(nf, ng, s_red);
  if (threadIdx.x == 0) {
    atomicAdd(&a.norms[2 * w], static_cast<double>(nf));
    atomicAdd(&a.norms[2 * w + 1], static_cast<double>(ng));
  }
  // the cross power is Hermitian (P(-k) = conj P(k)), so the mirror row's inverse
  // transform is the conjugate of row u's: only the even lines are transformed back
  float2* R = fft_lines<true>(Y, X, L, lines / 2, 2 * L, 1, a.tw_pow2);
  for (int e = threadIdx.x; e < lines * L; e += kLineThreads) {
    const int line = e >> lg, y = e & (L - 1);
    const int u = u0 + (line >> 1);
    if (u >= nunits) continue;
    if ((line & 1) && (u == 0 || 2 * u == L)) continue;   // a self-paired row is written once
    const int row = (line & 1) ? (L - u) & (L - 1) : u;
    const float2 r = R[fsl((line & ~1) * L + y)];
    base[static_cast<int64_t>(row) * L + y] = (line & 1) ? make_float2(r.x, -r.y) : r;
  }
}

// Inverse transform of the rows along kx and the per-window arg-max of R. TR: the work
// buffer holds the transposed layout (work[w][kx][y]), read in runs of kTrRun rows.
template <bool TR>
__global__ void __launch_bounds__(kLineThreads, 3) fftcc_rows_inv_kernel(FftccArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = a.L;
  const int rows = kLineElems / L;
  float2* P = reinterpret_cast<float2*>(smem_raw);      // element e at slot fsl(e)
  float2* Q = P + fft_slots(kLineElems);
  __shared__ unsigned long long s_key[kLineThreads / 32];
  const int64_t w = blockIdx.x;
  if (!window_ok(a.org[w], L, a.W, a.H)) return;
  const int y0 = blockIdx.y * rows;
  if (TR) {
    const int lg = __ffs(L) - 1;
    const float2* base = a.work + w * static_cast<int64_t>(L) * L + y0;
    for (int it = threadIdx.x; it < (rows / kTrRun) * L; it += kLineThreads) {
      const int kx = it & (L - 1), r = kTrRun * (it >> lg);
      const float4* sp = reinterpret_cast<const float4*>(base + static_cast<int64_t>(kx) * L + r);
      float4 v[kTrRun / 2];
#pragma unroll
      for (int i = 0; i < kTrRun / 2; ++i) v[i] = sp[i];
#pragma unroll
      for (int i = 0; i < kTrRun / 2; ++i) {
        P[fsl((r + 2 * i) * L + kx)] = make_float2(v[i].x, v[i].y);
        P[fsl((r + 2 * i + 1) * L + kx)] = make_float2(v[i].z, v[i].w);
      }
    }
  } else {
    const float2* src = a.work + w * static_cast<int64_t>(L) * L + static_cast<int64_t>(y0) * L;
    for (int e = threadIdx.x; e < rows * L; e += kLineThreads) P[fsl(e)] = src[e];
  }
  __syncthreads();
  unsigned long long best = 0ull;
  if (rows >= 2) {
    // every row transforms back to real values: rows 2l and 2l + 1 go through one
    // transform as row 2l + i row 2l + 1, whose result holds them as real and
    // imaginary parts
    const int lg = __ffs(L) - 1;
    for (int e = threadIdx.x; e < (rows / 2) * L; e += kLineThreads) {
      const int l = e >> lg, x = e & (L - 1);
      const float2 p0 = P[fsl(2 * l * L + x)], p1 = P[fsl((2 * l + 1) * L + x)];
      Q[fsl(e)] = make_float2(p0.x - p1.y, p0.y + p1.x);
    }
    __syncthreads();
    const float2* R = fft_lines<true>(Q, P, L, rows / 2, L, 1, a.tw_pow2);
    for (int e = threadIdx.x; e < (rows / 2) * L; e += kLineThreads) {
      const int l = e >> lg, x = e & (L - 1);
      const float2 v = R[fsl(e)];
      const unsigned long long k0 = peak_key(v.x, (y0 + 2 * l) * L + x), k1 = peak_key(v.y, (y0 + 2 * l + 1) * L + x);
      best = k0 > best ? k0 : best;
      best = k1 > best ? k1 : best;
    }
  } else {
    const float2* R = fft_lines<true>(P, Q, L, rows, L, 1, a.tw_pow2);
    for (int e = threadIdx.x; e < rows * L; e += kLineThreads) {
      const unsigned long long k = peak_key(R[fsl(e)].x, y0 * L + e);
      best = k > best ? k : best;
    }
  }
  best = block_max_key(best, s_key);
  if (threadIdx.x == 0) atomicMax(&a.keys[w], best);
}

__global__ void fftcc_finish_kernel(FftccArgs a) {
  const int64_t w = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (w >= a.n) return;
  const int4 o = a.org[w];
  const int L = a.L;
  if (!window_ok(o, L, a.W, a.H)) {
    a.u[w] = 0.f;
    a.v[w] = 0.f;
    a.peak[w] = 0.f;
    return;
  }
  const bool flat = !a.nonflat[2 * w] || !a.nonflat[2 * w + 1];
  const unsigned long long key = a.keys[w];
  const int e = flat ? 0 : key_index(key);
  const int ky = e / L, kx = e - ky * L;
  a.u[w] = static_cast<float>(o.z - o.x + shift_of_peak(kx, L));
  a.v[w] = static_cast<float>(o.w - o.y + shift_of_peak(ky, L));
  const double den = sqrt(a.norms[2 * w] * a.norms[2 * w + 1]);
  a.peak[w] = flat || !(den > 0.0) ? 0.f : static_cast<float>(static_cast<double>(key_value(key)) / den);
}

// ---------------------------------------------------------------- level set-up
// Reference and deformed origins of every window of a level (readings of the
// initialiser: tiles of side L, or the subsets of the correlation grid, each moved
// by the previous level's field interpolated bilinearly and rounded, clamped into
// the image). The arithmetic is FP64 without contraction, as in the definition.
__global__ void fftcc_origins_kernel(FftLevelArgs a) {
  const int64_t w = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (w >= static_cast<int64_t>(a.nx) * a.ny) return;
  const int i = static_cast<int>(w % a.nx), j = static_cast<int>(w / a.nx);
  if (a.roi_ok && !a.roi_ok[w]) {
    a.org[w] = make_int4(-1, -1, -1, -1);
    return;
  }
  int x0, y0, cx, cy;
  if (a.grid) {
    cx = a.r + i * a.step;
    cy = a.r + j * a.step;
    x0 = cx - a.r;
    y0 = cy - a.r;
  } else {
    x0 = i * a.L;
    y0 = j * a.L;
    cx = x0 + a.L / 2;
    cy = y0 + a.L / 2;
  }
  int gu = 0, gv = 0;
  if (a.pu) {
    const double c0 = a.pc0, st = a.pstep;
    double tx = __ddiv_rn(__dsub_rn(static_cast<double>(cx), c0), st);
    double ty = __ddiv_rn(__dsub_rn(static_cast<double>(cy), c0), st);
    tx = fmin(fmax(tx, 0.0), static_cast<double>(a.pnx - 1));
    ty = fmin(fmax(ty, 0.0), static_cast<double>(a.pny - 1));
    int i0 = static_cast<int>(floor(tx)), j0 = static_cast<int>(floor(ty));
    i0 = min(i0, max(a.pnx - 2, 0));
    j0 = min(j0, max(a.pny - 2, 0));
    const int i1 = min(i0 + 1, a.pnx - 1), j1 = min(j0 + 1, a.pny - 1);
    const double fx = __dsub_rn(tx, static_cast<double>(i0)), fy = __dsub_rn(ty, static_cast<double>(j0));
    auto lerp2 = [&](const float* F) {
      const double f00 = F[static_cast<int64_t>(j0) * a.pnx + i0], f01 = F[static_cast<int64_t>(j0) * a.pnx + i1];
      const double f10 = F[static_cast<int64_t>(j1) * a.pnx + i0], f11 = F[static_cast<int64_t>(j1) * a.pnx + i1];
      const double top = __dadd_rn(__dmul_rn(__dsub_rn(1.0, fx), f00), __dmul_rn(fx, f01));
      const double bot = __dadd_rn(__dmul_rn(__dsub_rn(1.0, fx), f10), __dmul_rn(fx, f11));
      return __dadd_rn(__dmul_rn(__dsub_rn(1.0, fy), top), __dmul_rn(fy, bot));
    };
    gu = static_cast<int>(floor(__dadd_rn(lerp2(a.pu), 0.5)));
    gv = static_cast<int>(floor(__dadd_rn(lerp2(a.pv), 0.5)));
  }
  const int gx0 = min(max(x0 + gu, 0), a.W - a.L);
  const int gy0 = min(max(y0 + gv, 0), a.H - a.L);
  a.org[w] = make_int4(x0, y0, gx0, gy0);
}

// ---------------------------------------------------------------- MAD removal
__device__ double median_sorted(const double* s, int n) {
  return (n & 1) ? s[n / 2] : __ddiv_rn(__dadd_rn(s[n / 2 - 1], s[n / 2]), 2.0);
}
__device__ void sort_small(double* s, int n) {
  for (int i = 1; i < n; ++i) {
    const double v = s[i];
    int j = i - 1;
    while (j >= 0 && s[j] > v) {
      s[j + 1] = s[j];
      --j;
    }
    s[j + 1] = v;
  }
}

__global__ void mad_kernel(MadArgs a) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= static_cast<int64_t>(a.nx) * a.ny) return;
  const int i = static_cast<int>(q % a.nx), j = static_cast<int>(q / a.nx);
  const double uq = a.u[q], vq = a.v[q];
  uint8_t rep = 0;
  double ou = uq, ov = vq;
  const bool valid = a.valid ? a.valid[q] != 0 : true;
  if (valid && a.tau > 0.0) {
    double su[9], sv[9];
    int n = 0;
    for (int dj = -1; dj <= 1; ++dj) {
      const int jj = j + dj;
      if (jj < 0 || jj >= a.ny) continue;
      for (int di = -1; di <= 1; ++di) {
        const int ii = i + di;
        if (ii < 0 || ii >= a.nx) continue;
        const int64_t r = static_cast<int64_t>(jj) * a.nx + ii;
        if (a.valid && !a.valid[r]) continue;
        su[n] = a.u[r];
        sv[n] = a.v[r];
        ++n;
      }
    }
    sort_small(su, n);
    sort_small(sv, n);
    const double mu = median_sorted(su, n), mv = median_sorted(sv, n);
    double du[9], dv[9];
    for (int k = 0; k < n; ++k) {
      du[k] = fabs(__dsub_rn(su[k], mu));
      dv[k] = fabs(__dsub_rn(sv[k], mv));
    }
    sort_small(du, n);
    sort_small(dv, n);
    const double madu = median_sorted(du, n), madv = median_sorted(dv, n);
    const double lim_u = __dmul_rn(a.tau, __dadd_rn(__dmul_rn(1.4826, madu), a.eps));
    const double lim_v = __dmul_rn(a.tau, __dadd_rn(__dmul_rn(1.4826, madv), a.eps));
    if (fabs(__dsub_rn(uq, mu)) > lim_u || fabs(__dsub_rn(vq, mv)) > lim_v) {
      ou = mu;
      ov = mv;
      rep = 1;
    }
  }
  a.u_out[q] = static_cast<float>(ou);
  a.v_out[q] = static_cast<float>(ov);
  if (a.replaced) a.replaced[q] = rep;
}

// ---------------------------------------------------------------- twiddles
// tw[ns - 1 + k] = exp(-2 pi i k / (2 ns)) for ns = 1, 2, .., 2048 (4095 entries),
// then exp(-2 pi i t / L) for t < L (the odd table), from FP64 sincospi.
__global__ void twiddle_kernel(float2* tw, int L_odd) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < kFftTwiddlesPow2) {
    const int ns = 1 << (31 - __clz(e + 1));              // the largest power of two <= e + 1
    const int k = e + 1 - ns;
    double s, c;
    sincospi(-static_cast<double>(k) / ns, &s, &c);
    tw[e] = make_float2(static_cast<float>(c), static_cast<float>(s));
  } else if (e < kFftTwiddlesPow2 + L_odd) {
    const int t = e - kFftTwiddlesPow2;
    double s, c;
    sincospi(-2.0 * t / L_odd, &s, &c);
    tw[e] = make_float2(static_cast<float>(c), static_cast<float>(s));
  }
}

__global__ void fft_status_kernel(const uint8_t* roi_ok, uint8_t* status, int64_t n) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q < n) status[q] = (!roi_ok || roi_ok[q]) ? DIC_PT_OK : DIC_PT_NOT_IN_ROI;
}

size_t small_smem(int L, bool pow2) {
  if (pow2) return sizeof(float2) * (2 * static_cast<size_t>(fft_slots(L * L)) + L - 1);
  return sizeof(float2) * 3 * static_cast<size_t>(L) * L;
}

int blocks_for(int64_t n, int per_sm) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t cap = static_cast<int64_t>(sms) * per_sm;
  return static_cast<int>(n < cap ? (n > 0 ? n : 1) : cap);
}

}  // namespace

cudaError_t launch_twiddles(float2* tw, int L_odd, cudaStream_t s) {
  const int n = kFftTwiddlesPow2 + L_odd;
  twiddle_kernel<<<(n + 255) / 256, 256, 0, s>>>(tw, L_odd);
  return cudaGetLastError();
}

cudaError_t launch_fftcc_origins(const FftLevelArgs& a, cudaStream_t s) {
  const int64_t n = static_cast<int64_t>(a.nx) * a.ny;
  if (n == 0) return cudaSuccess;
  fftcc_origins_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fft_status(const uint8_t* roi_ok, uint8_t* status, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  fft_status_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(roi_ok, status, n);
  return cudaGetLastError();
}

cudaError_t launch_mad(const MadArgs& a, cudaStream_t s) {
  const int64_t n = static_cast<int64_t>(a.nx) * a.ny;
  if (n == 0) return cudaSuccess;
  mad_kernel<<<static_cast<unsigned>((n + 127) / 128), 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fftcc(const FftccArgs& a, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  const int L = a.L;
  const bool pow2 = (L & (L - 1)) == 0;
  if (L <= kTcP) {
    // windows up to 32: the DFT products on the tensor cores
    static const cudaError_t ok_tc = cudaFuncSetAttribute(fftcc_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          static_cast<int>(tc_smem()));
    if (ok_tc != cudaSuccess) return ok_tc;
    fftcc_tc_kernel<<<blocks_for((a.n + kTcWarps - 1) / kTcWarps, 1), kTcBlockThreads, tc_smem(), s>>>(a);
    return cudaGetLastError();
  }
  if (L <= kFftSmallMax) {
    const size_t smem = small_smem(L, pow2);
    if (pow2) {
      static const cudaError_t ok = cudaFuncSetAttribute(fftcc_small_kernel<true>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         static_cast<int>(small_smem(kFftSmallMax, true)));
      if (ok != cudaSuccess) return ok;
      // blocks per SM within 224 KB of shared memory (1 KB reserved per block)
      const int fit = static_cast<int>(224 * 1024 / (smem + 1024));
      const int per_sm = fit < 8 ? fit : 8;
      fftcc_small_kernel<true><<<blocks_for(a.n, per_sm > 0 ? per_sm : 1), kSmallThreads, smem, s>>>(a);
    } else {
      static const cudaError_t ok = cudaFuncSetAttribute(fftcc_small_kernel<false>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         static_cast<int>(small_smem(kFftSmallMax, false)));
      if (ok != cudaSuccess) return ok;
      const int per_sm = static_cast<int>(200 * 1024 / smem) < 8 ? static_cast<int>(200 * 1024 / smem) : 8;
      fftcc_small_kernel<false><<<blocks_for(a.n, 2 * (per_sm > 0 ? per_sm : 1)), kSmallThreads / 2, smem, s>>>(a);
    }
    return cudaGetLastError();
  }
  // large windows: a power of two in [128, 4096] (checked by the caller). Up to 512 the
  // row kernels write and read the work buffer transposed (runs of kTrRun rows), so the
  // two transpose kernels drop out; above, a block holds fewer rows (and four-row runs
  // measured slower than the transposes at 1024).
  const int line_bytes = static_cast<int>(2 * fft_slots(kLineElems) * sizeof(float2));
  static const cudaError_t ok1 = cudaFuncSetAttribute(fftcc_rows_fwd_kernel<false>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, line_bytes);
  static const cudaError_t ok1t = cudaFuncSetAttribute(fftcc_rows_fwd_kernel<true>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, line_bytes);
  static const cudaError_t ok2 = cudaFuncSetAttribute(fftcc_pairs_kernel,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      static_cast<int>(2 * fft_slots(2 * kLineElems) * sizeof(float2)));
  static const cudaError_t ok3 = cudaFuncSetAttribute(fftcc_rows_inv_kernel<false>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, line_bytes);
  static const cudaError_t ok3t = cudaFuncSetAttribute(fftcc_rows_inv_kernel<true>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, line_bytes);
  for (cudaError_t ok : {ok1, ok1t, ok2, ok3, ok3t})
    if (ok != cudaSuccess) return ok;
  cudaError_t e;
  if ((e = cudaMemsetAsync(a.nonflat, 0, sizeof(int32_t) * 2 * a.n, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.norms, 0, sizeof(double) * 2 * a.n, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.keys, 0, sizeof(unsigned long long) * a.n, s)) != cudaSuccess) return e;
  const unsigned nw = static_cast<unsigned>(a.n);
  const int rows = kLineElems / L;
  const bool tr = rows >= kTrRun;
  const size_t line_smem = static_cast<size_t>(line_bytes);
  const int T = L / kTransposeTile;
  if (tr) {
    fftcc_rows_fwd_kernel<true><<<dim3(nw, L / rows), kLineThreads, line_smem, s>>>(a);
  } else {
    fftcc_rows_fwd_kernel<false><<<dim3(nw, L / rows), kLineThreads, line_smem, s>>>(a);
    fftcc_transpose_kernel<<<dim3(nw, T * T), kTransposeTile * 8, 0, s>>>(a);
  }
  const int units = L <= kLineElems / 2 ? kLineElems / 2 / L : 1;
  const int nunits = L / 2 + 1;
  const size_t pair_smem = 2 * sizeof(float2) * fft_slots(2 * units * L);
  fftcc_pairs_kernel<<<dim3(nw, (nunits + units - 1) / units), kLineThreads, pair_smem, s>>>(a);
  if (tr) {
    fftcc_rows_inv_kernel<true><<<dim3(nw, L / rows), kLineThreads, line_smem, s>>>(a);
  } else {
    fftcc_transpose_kernel<<<dim3(nw, T * T), kTransposeTile * 8, 0, s>>>(a);
    fftcc_rows_inv_kernel<false><<<dim3(nw, L / rows), kLineThreads, line_smem, s>>>(a);
  }
  fftcc_finish_kernel<<<(nw + 255) / 256, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dic
