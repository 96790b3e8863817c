"""Fit the single-precision normal CDF / quantile polynomials used by the sweep kernel.

Writes normal_f32_coeffs.cuh beside this file.  Run: python fit_normal_f32.py

Upper tail: Phi(-y) = exp(-y^2/2) G(y) for y >= 0, with
G(y) = erfcx(y / sqrt 2) / 2 approximated as t Q(t), t = 1 / (1 + c y), Q a
degree-8 polynomial (weighted least squares iterated towards minimax relative
error by Lawson's method), fitted on y in [0, 40].

Quantile: Phi^{-1}(x) = sqrt(2) erfinv(2x - 1) and erfinv(v) = v P(w) with
w = -log(1 - v^2) = -log(4 x (1 - x)).  P is piecewise polynomial: degree 8
in w - 2.5 for w < 5, degree 7 in sqrt(w) - c1 for 5 <= w < 16, degree 6 in
sqrt(w) - c2 for 16 <= w <= 88 (x down to the smallest normal float).  A
branch-free variant for the paired sweep uses one tail piece instead:
P = sqrt(w) T(1/sqrt(w) - c3), T of degree 9, for 5 <= w <= 88.
The paired sweep (two evaluations per FP32x2 instruction) has its own,
shorter set, since its exponential is the hardware exp2 approximation
(relative error ~3e-6) anyway and the single-precision tolerances leave room:
G of degree 6 fitted on y in [0, 14] (beyond, the weight underflows) and the
central quantile piece of degree 6.  The tail quantile keeps degree 9: an
error in a deep conditional draw is amplified by the next limit (d log Phi(-y)
/ dy ~ -y), and degree 7 pushed log f past 1e-4 on deep-tail pairs.
The targets come from scipy.special (erfcx, ndtri) in double precision.
"""
import os

import numpy as np
from scipy import special

HERE = os.path.dirname(os.path.abspath(__file__))
F32_TINY = float(np.finfo(np.float32).tiny)


def lawson(V, target, iters=40):
    w = 1.0 / np.abs(target)
    W = np.ones_like(target)
    coef = None
    for _ in range(iters):
        coef, *_ = np.linalg.lstsq(V * (w * W)[:, None], target * w * W, rcond=None)
        err = np.abs(V @ coef - target) / np.abs(target)
        W = W * err
        W /= W.mean()
    return coef


def cheb_nodes(lo, hi, m=6000):
    k = np.arange(m)
    return 0.5 * (lo + hi) + 0.5 * (hi - lo) * np.cos(np.pi * (k + 0.5) / m)


def fit_tail(c=0.36, deg=8, ymax=40.0):
    tmin = 1.0 / (1.0 + c * ymax)
    t = cheb_nodes(tmin, 1.0)
    y = (1.0 / t - 1.0) / c
    Q = 0.5 * special.erfcx(y / np.sqrt(2.0)) / t
    return lawson(np.vander(t, deg + 1, increasing=True), Q)


def fit_quantile_piece(wlo, whi, use_sqrt, deg):
    if use_sqrt:
        s = cheb_nodes(np.sqrt(wlo), np.sqrt(whi))
        w = s * s
        cen = 0.5 * (np.sqrt(wlo) + np.sqrt(whi))
        v = s - cen
    else:
        w = cheb_nodes(wlo, whi)
        cen = 0.5 * (wlo + whi)
        v = w - cen
    y = np.sqrt(-np.expm1(-w))
    one_minus_y = np.exp(-w) / (1.0 + y)
    P = -special.ndtri(one_minus_y / 2.0) / np.sqrt(2.0) / y
    return cen, lawson(np.vander(v, deg + 1, increasing=True), P)


def fit_quantile_tail_inv(wlo, whi, deg):
    a, b = 1.0 / np.sqrt(whi), 1.0 / np.sqrt(wlo)
    v = cheb_nodes(a, b, 8000)
    w = 1.0 / (v * v)
    y = np.sqrt(-np.expm1(-w))
    one_minus_y = np.exp(-w) / (1.0 + y)
    P = -special.ndtri(one_minus_y / 2.0) / np.sqrt(2.0) / y
    cen = 0.5 * (a + b)
    return cen, lawson(np.vander(v - cen, deg + 1, increasing=True), P * v, iters=80)


def fmt(arr):
    return ", ".join(f"{float(np.float32(a)):.9e}f" for a in arr)


def main():
    c = 0.36
    q = fit_tail(c)
    wmax = -np.log(4.0 * F32_TINY) + 1.0
    c0, p0 = fit_quantile_piece(1e-12, 5.0, False, 8)
    c1, p1 = fit_quantile_piece(5.0, 16.0, True, 7)
    c2, p2 = fit_quantile_piece(16.0, wmax, True, 6)
    c3, p3 = fit_quantile_tail_inv(5.0, wmax, 9)
    cf = 0.36
    qf = fit_tail(cf, 6, 14.0)
    c0f, p0f = fit_quantile_piece(1e-12, 5.0, False, 6)
    text = f"""// Generated by fit_normal_f32.py (least-squares fits iterated towards minimax
// relative error); see that script for the forms.  Do not edit by hand.
#pragma once

namespace cfust {{
namespace nf32 {{

// Phi(-y) = exp(-y^2/2) * t * Q(t), t = 1 / (1 + TAIL_C y), y >= 0
constexpr float TAIL_C = {np.float32(c):.9e}f;
__device__ constexpr float TAIL_Q[9] = {{{fmt(q)}}};

// Phi^-1(x) = sqrt(2) (2x - 1) P(w), w = -log(4 x (1 - x))
constexpr float Q_W0 = {np.float32(c0):.9e}f;   // w < 5: P = poly(w - Q_W0)
__device__ constexpr float Q_P0[9] = {{{fmt(p0)}}};
constexpr float Q_S1 = {np.float32(c1):.9e}f;   // 5 <= w < 16: P = poly(sqrt(w) - Q_S1)
__device__ constexpr float Q_P1[8] = {{{fmt(p1)}}};
constexpr float Q_S2 = {np.float32(c2):.9e}f;   // w >= 16: P = poly(sqrt(w) - Q_S2)
__device__ constexpr float Q_P2[7] = {{{fmt(p2)}}};
constexpr float Q_U3 = {np.float32(c3):.9e}f;   // w >= 5 (branch-free form): P = sqrt(w) poly(1/sqrt(w) - Q_U3)
__device__ constexpr float Q_P3[10] = {{{fmt(p3)}}};

// Shorter set of the paired sweep (same forms)
constexpr float TAIL_CF = {np.float32(cf):.9e}f;
__device__ constexpr float TAIL_QF[7] = {{{fmt(qf)}}};
constexpr float Q_W0F = {np.float32(c0f):.9e}f;
__device__ constexpr float Q_P0F[7] = {{{fmt(p0f)}}};

}}  // namespace nf32
}}  // namespace cfust
"""
    with open(os.path.join(HERE, "normal_f32_coeffs.cuh"), "w") as f:
        f.write(text)
    print(text)


if __name__ == "__main__":
    main()
