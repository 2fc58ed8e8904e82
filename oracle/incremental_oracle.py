"""FP64 CPU oracle of incremental reference updating for image sequences (the
scheme the paper plans in Sec. 6 after Pan et al. 2012: the reference image evolves
through the sequence so that large strains stay within reach of the subset shape
function).

TEST INFRASTRUCTURE. This module is the plain, slow, obviously correct reference
that the CUDA library is checked against. Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import it; the library never does, and it shares
no code, table or constant with the library.

Readings (the paper names the scheme only; all of them are this oracle's):

  I1 Updates are explicit: after frame r the caller may make frame r the reference.
     The subset grid stays the same integer grid (reading R3) in every reference.
  I2 Every grid point Q of the first reference carries an accumulated warp
     (u_a, v_a, A_a) from frame 0 to the current reference (A = [[p2, p3], [p4, p5]],
     Eq. 5; rigid: A = 0), starting from the identity for the in-ROI points. A frame k
     correlated against reference r gives its total warp: x_r = X_Q + (u_a, v_a); the
     grid point q of reference r nearest to x_r (per axis, ties to the lower index)
     must exist and be accepted in frame k; its warp re-expanded at the offset
     x_r - x_q (reading R10) gives (d, A_i); then
         (u, v) = (u_a, v_a) + d,      I + A = (I + A_i)(I + A_a).
     Otherwise the point has no total in that frame (status NOT_REACHED). An update
     after frame r makes frame r's totals the new accumulated warps (points without
     one drop out for good).
  I3 The frame after an update starts every in-ROI point of the new reference from
     the identity warp, all in wave 0 (then reading R11 / R10 as usual); frame 1
     starts from the seeds.
  I4 Rigid and affine shape functions only: the composition of two quadratic warps
     of Eq. 5 is not a quadratic warp.
"""
from __future__ import annotations

import math

import numpy as np

from .dic_oracle import (AFFINE, NOT_IN_ROI, NOT_REACHED, N_PARAMS, OK, QUADRATIC, correlate, correlate_sequence,
                         grid, roi_points, transfer_warp, _propagate)


def gradient_matrix(p):
    """A of reading I2 from Eq. 5 parameters (zeros for the rigid shape function)."""
    p = np.asarray(p, dtype=np.float64)
    if len(p) < 6:
        return np.zeros((2, 2))
    return np.array([[p[2], p[3]], [p[4], p[5]]])


def compose(acc_uv, acc_A, inc_p, offset):
    """Reading I2: the increment re-expanded at offset, composed after the accumulated
    warp. Returns (u, v) and A."""
    q = transfer_warp(np.asarray(inc_p, dtype=np.float64), float(offset[0]), float(offset[1]))
    Ai = gradient_matrix(q)
    total_A = (np.eye(2) + Ai) @ (np.eye(2) + np.asarray(acc_A)) - np.eye(2)
    return (acc_uv[0] + q[0], acc_uv[1] + q[1]), total_A


def nearest_index(t, n):
    """Nearest integer to t, ties to the lower one; None outside [0, n)."""
    i = math.ceil(t - 0.5)
    return i if 0 <= i < n else None


def totals(acc, res, W, H, subset_size, subset_step, shape):
    """Reading I2 for every grid point: the total warps (frame 0 to the frame of res)."""
    xs, ys = grid(W, H, subset_size, subset_step)
    nx, ny = len(xs), len(ys)
    r = (subset_size - 1) // 2
    n = N_PARAMS[shape]
    npts = nx * ny
    out_p = np.zeros((npts, n))
    status = np.full(npts, NOT_REACHED, np.int32)
    status[acc["status"] == NOT_IN_ROI] = NOT_IN_ROI
    for Q in range(npts):
        if not acc["ok"][Q]:
            continue
        X, Y = xs[Q % nx], ys[Q // nx]
        xr, yr = X + acc["u"][Q], Y + acc["v"][Q]
        i = nearest_index((xr - r) / subset_step, nx)
        j = nearest_index((yr - r) / subset_step, ny)
        if i is None or j is None:
            continue
        q = j * nx + i
        if res["status"][q] != OK:
            continue
        (u, v), A = compose((acc["u"][Q], acc["v"][Q]), acc["A"][Q], res["p"][q], (xr - xs[i], yr - ys[j]))
        out_p[Q, 0], out_p[Q, 1] = u, v
        if n >= 6:
            out_p[Q, 2:6] = A[0, 0], A[0, 1], A[1, 0], A[1, 1]
        status[Q] = OK
    return dict(u=out_p[:, 0].copy(), v=out_p[:, 1].copy(), p=out_p, status=status, nx=nx, ny=ny)


def identity_acc(roi, W, H, subset_size, subset_step):
    inroi = roi_points(roi, W, H, subset_size, subset_step).ravel()
    n = len(inroi)
    return dict(u=np.zeros(n), v=np.zeros(n), A=np.zeros((n, 2, 2)), ok=inroi.copy(),
                status=np.where(inroi, OK, NOT_IN_ROI).astype(np.int32))


def correlate_incremental(frames, roi, subset_size, subset_step, shape, seeds, params=None, update_after=()):
    """Readings I1-I4 over frames[0] (the first reference) and frames[1:]. Returns, per
    frame k >= 1, (res_k, tot_k): the correlation against the current reference and the
    total warps from frame 0."""
    if shape == QUADRATIC:
        raise ValueError("reference updating needs a rigid or affine shape function (reading I4)")
    H, W = np.asarray(frames[0]).shape
    ref = frames[0]
    acc = identity_acc(roi, W, H, subset_size, subset_step)
    n = N_PARAMS[shape]
    out = []
    prev = None
    fresh = False
    for k in range(1, len(frames)):
        if prev is None:
            res = correlate(ref, frames[k], roi, subset_size, subset_step, shape, seeds, params)
        elif fresh:
            inroi = roi_points(roi, W, H, subset_size, subset_step).ravel()
            starts = {int(q): np.zeros(n) for q in np.flatnonzero(inroi)}
            res = _propagate(ref, frames[k], roi, subset_size, subset_step, shape, params, None, starts=starts)
        else:
            res = correlate_sequence(ref, frames[k], roi, subset_size, subset_step, shape, prev, params)
        tot = totals(acc, res, W, H, subset_size, subset_step, shape)
        out.append((res, tot))
        prev = res
        fresh = False
        if k in update_after:
            ok = tot["status"] == OK
            A = np.zeros((len(ok), 2, 2))
            if n >= 6:
                A[:, 0, 0], A[:, 0, 1], A[:, 1, 0], A[:, 1, 1] = (tot["p"][:, 2], tot["p"][:, 3], tot["p"][:, 4],
                                                                  tot["p"][:, 5])
            acc = dict(u=tot["u"].copy(), v=tot["v"].copy(), A=A, ok=ok,
                       status=np.where(acc["status"] == NOT_IN_ROI, NOT_IN_ROI, OK).astype(np.int32))
            ref = frames[k]
            fresh = True
    return out
