// Standard normal quantile Phi^-1(p) for the Gaussian part of Alg. 1.
//
// Our own approximation, written from the relation
// Phi^-1(p) = sqrt(2) erfinv(2p - 1) and the split of erfinv used by Giles
// ("Approximating the erfinv function", GPU Computing Gems, 2010): with
// x = 2p - 1 and w = -ln(1 - x^2) = -ln(4 p (1 - p)),
//   erfinv(x) = x P1(w)          for w < 5   (p in (0.0017, 0.9983))
//   erfinv(x) = x P2(sqrt(w))    otherwise.
// Here the logarithm is taken in base 2, w2 = -log2(4p - 4p^2) = w / ln 2
// (the hardware lg2, no conversion), and the factor sqrt(2) is part of the
// polynomials: Phi^-1(p) = x Q1(w2 - c1) for w2 < 5 / ln 2, else
// x Q2(sqrt(w2) - c2), Q1 and Q2 of degree 9 with coefficients fitted for
// this library by weighted least squares against the exact quantile.  For the
// uniforms the hash produces, p = (2m + 1) 2^-24, x is exact in FP32 and
// 4p - 4p^2 is rounded once (one fused multiply-add); lg2's error moves Q1 by
// less than 3e-8 relative; the result stays within 2.5e-7 relative (4.2e-8
// absolute for |z| < 1/4) of the exact quantile.
#pragma once

namespace glint {

__device__ __forceinline__ float normal_quantile(float p) {
    const float x = 2.f * p - 1.f;
    const float p4 = 4.f * p;
    float w2;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(w2) : "f"(fmaf(-p4, p, p4)));
    w2 = -w2;
    float P;
    if (w2 < 7.213475227f) {
        const float t = w2 - 3.606737614f;
        P = -4.593011249e-10f;
        P = fmaf(P, t, 1.750330991e-09f);
        P = fmaf(P, t, 5.068341480e-08f);
        P = fmaf(P, t, -5.430951546e-07f);
        P = fmaf(P, t, -1.123125344e-06f);
        P = fmaf(P, t, 7.127850404e-05f);
        P = fmaf(P, t, -5.900012329e-04f);
        P = fmaf(P, t, -2.838380402e-03f);
        P = fmaf(P, t, 2.417711467e-01f);
        P = fmaf(P, t, 2.123313427e+00f);
    } else {
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(w2));
        const float t = r - 3.603367329f;
        P = 3.712571197e-05f;
        P = fmaf(P, t, -1.050955761e-04f);
        P = fmaf(P, t, -3.455006663e-05f);
        P = fmaf(P, t, 7.061248762e-04f);
        P = fmaf(P, t, -2.025795635e-03f);
        P = fmaf(P, t, 3.860775614e-03f);
        P = fmaf(P, t, -6.235580891e-03f);
        P = fmaf(P, t, 9.259297512e-03f);
        P = fmaf(P, t, 1.179382324e+00f);
        P = fmaf(P, t, 4.006434441e+00f);
    }
    return P * x;
}

}  // namespace glint
