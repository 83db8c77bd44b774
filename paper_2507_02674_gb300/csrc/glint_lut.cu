// Microfacet tables over (mu_o, sqrt alpha): V = E_D / D_H, U = 1 - V and the
// split-sum albedo terms A, B.
//
// E_D(w_o) = int D(h) 1[h.w_o > 0] 1[n.w_i(h) > 0] dh is the visible reflecting
// microfacet area (Sec. 4 Eq. rtiblndf, via the change of variables of
// Sec. 3.2), D_H = int D(h) dh the total microfacet area (Sec. 3.2), and
// E_rho = F0 A + B the directional albedo of the split sum (Sec. 3.4
// Eq. rtibl) with Schlick's F and the height-correlated Smith G2.
//
// Integration variable: with u the GGX CDF in theta_h and s = sqrt(1 - u),
// D(h) dh = 2 sqrt(a^2 + (1-a^2) s^2) ds dphi / (2 pi) is bounded; phi runs over
// [0, pi) by the mirror symmetry of the configuration.  V and U integrate the
// validity indicator over phi in closed form (an arc) with a Q*Q-point
// midpoint rule in s, so no quadrature point sits on a discontinuity; A and B
// use a Q x Q midpoint rule in (s, phi), their integrand vanishing on the
// boundary of the valid set.  One block per node; each thread sums its points
// with compensated (Kahan) summation before the block reduction.
#include "glint_internal.cuh"

using glint::kPi;

namespace {

struct KahanSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

__device__ __forceinline__ float smith_lambda(float mu, float a2) {
    if (mu >= 1.f) return 0.f;
    float t2 = (1.f - mu * mu) / (mu * mu);
    return 0.5f * (-1.f + sqrtf(1.f + a2 * t2));
}

template <int NT>
__global__ void __launch_bounds__(NT) k_lut(float4 *__restrict__ lut, int n, int Q) {
    const int node = blockIdx.x;
    const int i = node % n;  // mu_o column
    const int j = node / n;  // sqrt(alpha) row
    const float mu = ((float)i + 0.5f) / (float)n;
    const float st = ((float)j + 0.5f) / (float)n;
    const float alpha = st * st;
    const float a2 = alpha * alpha;
    const float sv = sqrtf(fmaxf(1.f - mu * mu, 0.f));
    const float lam_o = smith_lambda(mu, a2);

    KahanSum s_all, s_valid, s_invalid, s_A, s_B;
    const int total = Q * Q;
    const float inv_total = 1.f / (float)total;
    for (int t = threadIdx.x; t < total; t += NT) {
        // V, U: point t of the Q*Q-point rule in s; the valid normals at this
        // theta_h form the arc cos(phi) > c* = -(mu / sin theta_o) cot(2 theta_h).
        {
            const float s = ((float)t + 0.5f) * inv_total;
            const float root2 = a2 + (1.f - a2) * s * s;
            const float w = 2.f * sqrtf(root2);
            float m;
            if (sv > 0.f) {
                const float cos2t = s * s - a2 * (1.f - s * s);
                const float sin2t = 2.f * s * alpha * sqrtf(1.f - s * s);
                const float cstar = -(mu / sv) * (cos2t / sin2t);
                m = acosf(fminf(fmaxf(cstar, -1.f), 1.f));
                s_valid.add(w * m);
                s_invalid.add(w * acosf(fminf(fmaxf(-cstar, -1.f), 1.f)));
            } else {
                m = (s * s - a2 * (1.f - s * s) > 0.f) ? kPi : 0.f;
                s_valid.add(w * m);
                s_invalid.add(w * (kPi - m));
            }
            s_all.add(w);
        }
        // A, B: point (a, b) of the Q x Q rule in (s, phi)
        const int a = t / Q, b = t % Q;
        const float s = ((float)a + 0.5f) / (float)Q;
        const float root = sqrtf(a2 + (1.f - a2) * s * s);
        const float w = 2.f * root;
        const float cos_h = s / root;
        const float sin_h = alpha * sqrtf(1.f - s * s) / root;
        const float phi = kPi * ((float)b + 0.5f) / (float)Q;
        const float vh = sv * sin_h * cosf(phi) + mu * cos_h;
        const float li_z = 2.f * vh * cos_h - mu;
        if (vh > 0.f && li_z > 0.f) {
            const float G2 = 1.f / (1.f + lam_o + smith_lambda(li_z, a2));
            const float om = 1.f - vh;
            const float om2 = om * om;
            const float Fc = om2 * om2 * om;
            const float g = G2 * vh / mu;
            s_A.add(w * (1.f - Fc) * g);
            s_B.add(w * Fc * g);
        }
    }
    __shared__ float red[5][NT];
    red[0][threadIdx.x] = s_all.s;
    red[1][threadIdx.x] = s_valid.s;
    red[2][threadIdx.x] = s_invalid.s;
    red[3][threadIdx.x] = s_A.s;
    red[4][threadIdx.x] = s_B.s;
    __syncthreads();
    for (int off = NT / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            for (int k = 0; k < 5; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float norm = 1.f / ((float)Q * (float)Q);
        lut[node] = make_float4(red[1][0] / (kPi * red[0][0]), red[2][0] / (kPi * red[0][0]), red[3][0] * norm,
                                red[4][0] * norm);
    }
}

}  // namespace

cudaError_t glint_launch_lut(float4 *lut, int n, int q, cudaStream_t s) {
    k_lut<256><<<n * n, 256, 0, s>>>(lut, n, q);
    return cudaGetLastError();
}
