// Generated by fit_normal_f32.py (least-squares fits iterated towards minimax
// relative error); see that script for the forms.  Do not edit by hand.
#pragma once

namespace cfust {
namespace nf32 {

// Phi(-y) = exp(-y^2/2) * t * Q(t), t = 1 / (1 + TAIL_C y), y >= 0
constexpr float TAIL_C = 3.600000143e-01f;
__device__ constexpr float TAIL_Q[9] = {1.436176449e-01f, 1.436823308e-01f, 1.240042746e-01f, 9.607081115e-02f, -4.999166704e-04f, 1.075929552e-01f, -2.238538563e-01f, 1.396627426e-01f, -3.027698584e-02f};

// Phi^-1(x) = sqrt(2) (2x - 1) P(w), w = -log(4 x (1 - x))
constexpr float Q_W0 = 2.500000000e+00f;   // w < 5: P = poly(w - Q_W0)
__device__ constexpr float Q_P0[9] = {1.501409411e+00f, 2.466407120e-01f, -4.177726340e-03f, -1.253693365e-03f, 2.186181955e-04f, -4.401304523e-06f, -3.533135668e-06f, 3.441411423e-07f, 2.888704920e-08f};
constexpr float Q_S1 = 3.118033886e+00f;   // 5 <= w < 16: P = poly(sqrt(w) - Q_S1)
__device__ constexpr float Q_P1[8] = {2.951328993e+00f, 1.003614783e+00f, 7.143120747e-03f, -5.344045814e-03f, 3.995609470e-03f, -2.799534472e-03f, 1.053906628e-03f, -1.923229320e-05f};
constexpr float Q_S2 = 6.662355900e+00f;   // w >= 16: P = poly(sqrt(w) - Q_S2)
__device__ constexpr float Q_P2[7] = {6.528412819e+00f, 1.008939028e+00f, -5.080039264e-04f, 6.837136652e-07f, 6.515165296e-06f, -3.699315812e-06f, 8.880823543e-07f};
constexpr float Q_U3 = 2.772277594e-01f;   // w >= 5 (branch-free form): P = sqrt(w) poly(1/sqrt(w) - Q_U3)
__device__ constexpr float Q_P3[10] = {9.546209574e-01f, -1.925693303e-01f, 1.252948493e-01f, 5.648402572e-01f, 8.162746429e-01f, 1.152263451e+01f, 9.296464920e+00f, -1.601646576e+02f, -2.552538452e+02f, 1.114506958e+03f};

// Shorter set of the paired sweep (same forms)
constexpr float TAIL_CF = 3.600000143e-01f;
__device__ constexpr float TAIL_QF[7] = {1.437126100e-01f, 1.417795271e-01f, 1.396742910e-01f, 2.669101395e-02f, 1.807190627e-01f, -1.795689166e-01f, 4.699178413e-02f};
constexpr float Q_W0F = 2.500000000e+00f;
__device__ constexpr float Q_P0F[7] = {1.501409888e+00f, 2.466495484e-01f, -4.178334959e-03f, -1.265231404e-03f, 2.182244789e-04f, -6.660533813e-07f, -3.280813644e-06f};

}  // namespace nf32
}  // namespace cfust
