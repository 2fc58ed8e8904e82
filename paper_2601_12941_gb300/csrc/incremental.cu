// Incremental reference updating for image sequences (planned in Sec. 6 after Pan et
// al. 2012): every grid point of the first reference carries its warp from frame 0 to
// the current reference; a frame correlated against the current reference gives the
// point's total warp by composing the increment, taken at the point's current position
// from the nearest accepted grid point of the current reference (re-expanded there),
// after the accumulated warp:
//     (u, v) = (u_a, v_a) + d,      I + A = (I + A_i)(I + A_a),
// A the displacement gradient [[p2, p3], [p4, p5]] of Eq. 5 (zero for the rigid shape).
#include <math.h>

#include "dic_internal.cuh"

namespace dic {
namespace {

// nearest integer to t, ties to the lower one; -1 outside [0, n)
__device__ __forceinline__ int nearest_index(double t, int n) {
  const double i = ceil(t - 0.5);
  return (i >= 0.0 && i < static_cast<double>(n)) ? static_cast<int>(i) : -1;
}

__global__ void totals_kernel(TotalArgs a) {
  const int64_t n = static_cast<int64_t>(a.nx) * a.ny;
  for (int64_t Q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; Q < n;
       Q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int np = a.nparams;
    double* tp = a.tot_p + Q * np;
    for (int c = 0; c < np; ++c) tp[c] = 0.0;
    a.tot_u[Q] = 0.0;
    a.tot_v[Q] = 0.0;
    const bool in_roi = !(a.roi_ok && !a.roi_ok[Q]);
    uint8_t st = in_roi ? DIC_PT_NOT_REACHED : DIC_PT_NOT_IN_ROI;
    const bool acc_ok = in_roi && (a.identity || a.acc_ok[Q]);
    double ua = 0.0, va = 0.0, a00 = 0.0, a01 = 0.0, a10 = 0.0, a11 = 0.0;
    if (acc_ok && !a.identity) {
      ua = a.acc_u[Q];
      va = a.acc_v[Q];
      a00 = a.acc_A[4 * Q];
      a01 = a.acc_A[4 * Q + 1];
      a10 = a.acc_A[4 * Q + 2];
      a11 = a.acc_A[4 * Q + 3];
    }
    double u = 0.0, v = 0.0, t00 = 0.0, t01 = 0.0, t10 = 0.0, t11 = 0.0;
    if (acc_ok) {
      const int i = static_cast<int>(Q % a.nx), j = static_cast<int>(Q / a.nx);
      const double X = a.r + static_cast<double>(i) * a.step, Y = a.r + static_cast<double>(j) * a.step;
      const double xr = X + ua, yr = Y + va;
      const int iq = a.identity ? i : nearest_index((xr - a.r) / a.step, a.nx);
      const int jq = a.identity ? j : nearest_index((yr - a.r) / a.step, a.ny);
      if (iq >= 0 && jq >= 0) {
        const int64_t q = static_cast<int64_t>(jq) * a.nx + iq;
        if (a.status[q] == DIC_PT_OK) {
          const double* p = a.p + q * np;
          const double dx = xr - (a.r + static_cast<double>(iq) * a.step);
          const double dy = yr - (a.r + static_cast<double>(jq) * a.step);
          double d0 = p[0], d1 = p[1], i00 = 0.0, i01 = 0.0, i10 = 0.0, i11 = 0.0;
          if (np >= 6) {
            i00 = p[2];
            i01 = p[3];
            i10 = p[4];
            i11 = p[5];
            d0 = p[0] + p[2] * dx + p[3] * dy;
            d1 = p[1] + p[4] * dx + p[5] * dy;
          }
          u = ua + d0;
          v = va + d1;
          // (I + A_i)(I + A_a) - I = A_i + A_a + A_i A_a
          t00 = i00 + a00 + (i00 * a00 + i01 * a10);
          t01 = i01 + a01 + (i00 * a01 + i01 * a11);
          t10 = i10 + a10 + (i10 * a00 + i11 * a10);
          t11 = i11 + a11 + (i10 * a01 + i11 * a11);
          st = DIC_PT_OK;
          a.tot_u[Q] = u;
          a.tot_v[Q] = v;
          tp[0] = u;
          tp[1] = v;
          if (np >= 6) {
            tp[2] = t00;
            tp[3] = t01;
            tp[4] = t10;
            tp[5] = t11;
          }
          // no accumulated warp yet: the total is the point's own warp, whatever the shape
          if (a.identity)
            for (int c = 6; c < np; ++c) tp[c] = p[c];
        }
      }
    }
    a.tot_status[Q] = st;
    if (a.update) {
      a.acc_ok[Q] = st == DIC_PT_OK ? 1 : 0;
      a.acc_u[Q] = u;
      a.acc_v[Q] = v;
      a.acc_A[4 * Q] = t00;
      a.acc_A[4 * Q + 1] = t01;
      a.acc_A[4 * Q + 2] = t10;
      a.acc_A[4 * Q + 3] = t11;
    }
  }
}

// After an update every in-ROI point of the new reference starts the next sequence
// frame from the identity warp, in wave 0.
__global__ void identity_start_kernel(PointArrays pa, int nparams, const uint8_t* roi_ok) {
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < pa.n;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const bool in_roi = !(roi_ok && !roi_ok[q]);
    pa.u[q] = 0.0;
    pa.v[q] = 0.0;
    for (int c = 0; c < nparams; ++c) pa.p[q * nparams + c] = 0.0;
    pa.status[q] = in_roi ? DIC_PT_OK : DIC_PT_NOT_IN_ROI;
  }
}

unsigned blocks_of(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return static_cast<unsigned>(b < 8192 ? (b > 0 ? b : 1) : 8192);
}

}  // namespace

cudaError_t launch_totals(const TotalArgs& a, cudaStream_t s) {
  totals_kernel<<<blocks_of(static_cast<int64_t>(a.nx) * a.ny), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_identity_start(const PointArrays& pa, int nparams, const uint8_t* roi_ok, cudaStream_t s) {
  identity_start_kernel<<<blocks_of(pa.n), 256, 0, s>>>(pa, nparams, roi_ok);
  return cudaGetLastError();
}

}  // namespace dic
