/*
 * Device renderer of seeded synthetic speckle images (input generation only;
 * it is not part of the correlation library). One 256-thread block renders a
 * 32x32 tile exactly as the host renderer does: reference-frame coordinates,
 * their bounding box, a shared-memory table of the dots of the cells that can
 * reach the tile, then the per-pixel sum (the coordinates are recomputed there) in the fixed order of syn_speckle_sum.
 * Built with --fmad=false so its doubles match the host renderer's.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "speckle.h"

#define TILE 32
#define NT 256
#define TABLE_BYTES (40 * 1024)

enum { SYN_OUT_U8 = 0, SYN_OUT_U16 = 1, SYN_OUT_F32 = 2, SYN_OUT_F64 = 3 };

__global__ void __launch_bounds__(NT) syn_render_kernel(syn_speckle sp, syn_field fd,
                                                        syn_intensity it, int64_t W, int64_t H,
                                                        int out_kind, void* out,
                                                        int64_t row_stride_bytes) {
  __shared__ double red[4][NT / 32];
  __shared__ __align__(16) unsigned char table[TABLE_BYTES];
  __shared__ int64_t range[4];
  __shared__ int use_table;

  const int64_t tx0 = (int64_t)blockIdx.x * TILE, ty0 = (int64_t)blockIdx.y * TILE;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double xlo = 1e300, xhi = -1e300, ylo = 1e300, yhi = -1e300;
  for (int e = tid; e < TILE * TILE; e += NT) {
    int64_t x = tx0 + (e % TILE), y = ty0 + (e / TILE);
    double Xp = 0.0, Yp = 0.0;
    if (x < W && y < H) {
      syn_inverse_map(&fd, (double)x, (double)y, &Xp, &Yp);
      xlo = fmin(xlo, Xp);
      xhi = fmax(xhi, Xp);
      ylo = fmin(ylo, Yp);
      yhi = fmax(yhi, Yp);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    xlo = fmin(xlo, __shfl_xor_sync(0xffffffffu, xlo, o));
    xhi = fmax(xhi, __shfl_xor_sync(0xffffffffu, xhi, o));
    ylo = fmin(ylo, __shfl_xor_sync(0xffffffffu, ylo, o));
    yhi = fmax(yhi, __shfl_xor_sync(0xffffffffu, yhi, o));
  }
  if (lane == 0) {
    red[0][warp] = xlo;
    red[1][warp] = xhi;
    red[2][warp] = ylo;
    red[3][warp] = yhi;
  }
  __syncthreads();
  const int kmax = syn_kmax(&sp);
  if (tid == 0) {
    for (int w = 1; w < NT / 32; ++w) {
      xlo = fmin(xlo, red[0][w]);
      xhi = fmax(xhi, red[1][w]);
      ylo = fmin(ylo, red[2][w]);
      yhi = fmax(yhi, red[3][w]);
    }
    int64_t i0, i1, j0, j1;
    syn_cell_range(&sp, xlo, xhi, ylo, yhi, &i0, &i1, &j0, &j1);
    range[0] = i0;
    range[1] = i1;
    range[2] = j0;
    range[3] = j1;
    int64_t ncell = (i1 - i0 + 1) * (j1 - j0 + 1);
    int64_t need = ncell * (int64_t)sizeof(int) + 16 + ncell * kmax * (int64_t)sizeof(syn_dotrec);
    use_table = need <= TABLE_BYTES;
  }
  __syncthreads();
  const int64_t i0 = range[0], i1 = range[1], j0 = range[2], j1 = range[3];
  const int64_t ncx = i1 - i0 + 1;
  const int64_t ncell = ncx * (j1 - j0 + 1);
  int* counts = reinterpret_cast<int*>(table);
  size_t dots_off = ((size_t)ncell * sizeof(int) + 15) & ~(size_t)15;
  syn_dotrec* dots = reinterpret_cast<syn_dotrec*>(table + dots_off);
  if (use_table) {
    for (int64_t e = tid; e < ncell; e += NT)
      syn_fill_cell(&sp, i0 + (e % ncx), j0 + (e / ncx), kmax, &counts[e], &dots[e * kmax]);
  }
  __syncthreads();
  for (int e = tid; e < TILE * TILE; e += NT) {
    int64_t x = tx0 + (e % TILE), y = ty0 + (e / TILE);
    if (x >= W || y >= H) continue;
    double Xp, Yp;
    syn_inverse_map(&fd, (double)x, (double)y, &Xp, &Yp);
    double S = use_table ? syn_speckle_sum_table(&sp, counts, dots, kmax, i0, j0, (int)ncx, Xp, Yp)
                         : syn_speckle_sum(&sp, Xp, Yp);
    double I = syn_gray(&it, S) + syn_pixel_noise(&it, x, y, W);
    char* row = reinterpret_cast<char*>(out) + y * row_stride_bytes;
    if (out_kind == SYN_OUT_U8)
      reinterpret_cast<uint8_t*>(row)[x] = (uint8_t)syn_quantise(I, it.gray_max);
    else if (out_kind == SYN_OUT_U16)
      reinterpret_cast<uint16_t*>(row)[x] = (uint16_t)syn_quantise(I, it.gray_max);
    else if (out_kind == SYN_OUT_F32)
      reinterpret_cast<float*>(row)[x] = (float)I;
    else
      reinterpret_cast<double*>(row)[x] = I;
  }
}

extern "C" int syn_render_gpu(const syn_speckle* sp, const syn_field* fd, const syn_intensity* it,
                              int64_t W, int64_t H, int out_kind, void* out,
                              int64_t row_stride_bytes, void* stream) {
  if (W <= 0 || H <= 0 || out == nullptr) return -1;
  dim3 grid((unsigned)((W + TILE - 1) / TILE), (unsigned)((H + TILE - 1) / TILE));
  syn_render_kernel<<<grid, NT, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      *sp, *fd, *it, W, H, out_kind, out, row_stride_bytes);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : -(int)e;
}
