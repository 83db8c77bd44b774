// Standard normal quantile Phi^-1(p) for the Gaussian part of Alg. 1.
//
// Our own approximation, written from the relation
// Phi^-1(p) = sqrt(2) erfinv(2p - 1) and the split of erfinv used by Giles
// ("Approximating the erfinv function", GPU Computing Gems, 2010): with
// x = 2p - 1 and w = -ln(1 - x^2) = -ln(4 p (1 - p)),
//   erfinv(x) = x P1(w - 2.5)          for w < 5   (p in (0.0017, 0.9983))
//   erfinv(x) = x P2(sqrt(w) - 3)      otherwise,
// P1, P2 of degree 9 with coefficients fitted for this library by weighted
// least squares against the exact erfinv.  For the uniforms the hash produces,
// p = (2m + 1) 2^-24, x and 1 - p are exact in FP32; w uses the hardware
// logarithm (__logf), whose error moves P by less than 1.5e-7 relative; the
// result stays within 2.3e-7 relative (4e-8 absolute for |z| < 1/4) of the
// exact quantile.
#pragma once

namespace glint {

__device__ __forceinline__ float normal_quantile(float p) {
    const float x = 2.f * p - 1.f;
    const float w = -__logf(4.f * p * (1.f - p));
    float P;
    if (w < 5.f) {
        const float t = w - 2.5f;
        P = -8.627814907e-09f;
        P = fmaf(P, t, 2.224710549e-08f);
        P = fmaf(P, t, 4.639533415e-07f);
        P = fmaf(P, t, -3.451754537e-06f);
        P = fmaf(P, t, -4.953121788e-06f);
        P = fmaf(P, t, 2.183071483e-04f);
        P = fmaf(P, t, -1.252760063e-03f);
        P = fmaf(P, t, -4.177347291e-03f);
        P = fmaf(P, t, 2.466402948e-01f);
        P = fmaf(P, t, 1.501409411e+00f);
    } else {
        const float t = sqrtf(w) - 3.f;
        P = 1.319046423e-04f;
        P = fmaf(P, t, -3.114754509e-04f);
        P = fmaf(P, t, -8.706868539e-05f);
        P = fmaf(P, t, 1.487785368e-03f);
        P = fmaf(P, t, -3.579203971e-03f);
        P = fmaf(P, t, 5.686123855e-03f);
        P = fmaf(P, t, -7.641223725e-03f);
        P = fmaf(P, t, 9.445316158e-03f);
        P = fmaf(P, t, 1.001675129e+00f);
        P = fmaf(P, t, 2.832976818e+00f);
    }
    return 1.41421356f * (P * x);
}

}  // namespace glint
