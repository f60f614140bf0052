// QCP root for the MD kernel (shared by the FP32 pair kernel and the
// tensor-core estimate): Horn's 4x4 quaternion matrix N of the scaled 3x3
// correlation S = H / E0 (E0 = (G_x + G_y) / 2), the coefficients of its
// characteristic polynomial lambda^4 + c2 lambda^2 + c1 lambda + c0
// (c2 = -2 |S|_F^2, c1 = -8 det S, c0 = det N; Theobald 2005), and its largest
// root by Newton's method from the upper bound 1.
#pragma once

#include <cuda_runtime.h>

namespace kkm {

__device__ __forceinline__ float det3(float a, float b, float c, float d, float e, float f, float g,
                                      float h, float i) {
  return a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g);
}

// Minor of the symmetric 4x4 matrix m with row r and column c removed.
__device__ __forceinline__ float minor4(const float m[4][4], int r, int c) {
  int rr[3], cc[3];
  int k = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (q != r) rr[k++] = q;
  k = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (q != c) cc[k++] = q;
  return det3(m[rr[0]][cc[0]], m[rr[0]][cc[1]], m[rr[0]][cc[2]], m[rr[1]][cc[0]], m[rr[1]][cc[1]],
              m[rr[1]][cc[2]], m[rr[2]][cc[0]], m[rr[2]][cc[1]], m[rr[2]][cc[2]]);
}

// Cofactor row r of m (the r-th column of its adjugate).
template <int R>
__device__ __forceinline__ void cofactor_row(const float m[4][4], float v[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) v[c] = (((R + c) & 1) ? -1.f : 1.f) * minor4(m, R, c);
}

// Builds N (into m) from H scaled by 1 / E0 and the coefficients c2, c1, c0
// of its characteristic polynomial (its roots are <= 1 in these units).
__device__ __forceinline__ void qcp_coeffs(const float H[9], float E0, float m[4][4], float& c2, float& c1,
                                           float& c0) {
  const float inv = 1.0f / E0;
  const float Sxx = H[0] * inv, Sxy = H[1] * inv, Sxz = H[2] * inv;
  const float Syx = H[3] * inv, Syy = H[4] * inv, Syz = H[5] * inv;
  const float Szx = H[6] * inv, Szy = H[7] * inv, Szz = H[8] * inv;
  m[0][0] = Sxx + Syy + Szz;
  m[0][1] = Syz - Szy;
  m[0][2] = Szx - Sxz;
  m[0][3] = Sxy - Syx;
  m[1][1] = Sxx - Syy - Szz;
  m[1][2] = Sxy + Syx;
  m[1][3] = Szx + Sxz;
  m[2][2] = -Sxx + Syy - Szz;
  m[2][3] = Syz + Szy;
  m[3][3] = -Sxx - Syy + Szz;
  m[1][0] = m[0][1]; m[2][0] = m[0][2]; m[3][0] = m[0][3];
  m[2][1] = m[1][2]; m[3][1] = m[1][3]; m[3][2] = m[2][3];
  c2 = -2.0f * (Sxx * Sxx + Sxy * Sxy + Sxz * Sxz + Syx * Syx + Syy * Syy + Syz * Syz +
                            Szx * Szx + Szy * Szy + Szz * Szz);
  c1 = -8.0f * det3(Sxx, Sxy, Sxz, Syx, Syy, Syz, Szx, Szy, Szz);
  // det N by expansion in complementary 2x2 minors of rows (0,1) and (2,3)
  const float s0 = m[0][0] * m[1][1] - m[1][0] * m[0][1], s1 = m[0][0] * m[1][2] - m[1][0] * m[0][2];
  const float s2 = m[0][0] * m[1][3] - m[1][0] * m[0][3], s3 = m[0][1] * m[1][2] - m[1][1] * m[0][2];
  const float s4 = m[0][1] * m[1][3] - m[1][1] * m[0][3], s5 = m[0][2] * m[1][3] - m[1][2] * m[0][3];
  const float t5 = m[2][2] * m[3][3] - m[3][2] * m[2][3], t4 = m[2][1] * m[3][3] - m[3][1] * m[2][3];
  const float t3 = m[2][1] * m[3][2] - m[3][1] * m[2][2], t2 = m[2][0] * m[3][3] - m[3][0] * m[2][3];
  const float t1 = m[2][0] * m[3][2] - m[3][0] * m[2][2], t0 = m[2][0] * m[3][1] - m[3][0] * m[2][1];
  c0 = s0 * t5 - s1 * t4 + s2 * t3 + s3 * t2 - s4 * t1 + s5 * t0;
}

// The largest root lambda of N's characteristic polynomial, scaled by 1 / E0
// (so lambda <= 1), by Newton's method from the upper bound 1.
__device__ __forceinline__ float qcp_lambda(const float H[9], float E0, float m[4][4]) {
  float c2, c1, c0;
  qcp_coeffs(H, E0, m, c2, c1, c0);
  // Newton from the upper bound 1 (= (Gx+Gy)/2 after scaling)
  float lam = 1.0f;
  for (int it = 0; it < 60; ++it) {
    const float l2 = lam * lam;
    const float P = ((l2 + c2) * lam + c1) * lam + c0;
    const float dP = (4.0f * l2 + 2.0f * c2) * lam + c1;
    if (!(dP != 0.0f)) break;
    const float dl = P / dP;
    lam -= dl;
    if (fabsf(dl) <= 1e-7f * fabsf(lam)) break;
  }
  return lam;
}

// True if the pair is certainly far: rmsd^2 > r2_far, i.e. the largest root
// of the characteristic polynomial lies below x = 1 - n r2_far / (G_x + G_y).
// Sufficient test without root iteration: P(x) > 0 and its first three
// derivatives > 0 at x (the third is 24 x > 0), since then P(x + t) > 0 for
// every t >= 0 (Taylor expansion; the fourth derivative is 24).
__device__ __forceinline__ bool qcp_certainly_far(const float H[9], float Gx, float Gy, float n_r2_far) {
  const float E0 = 0.5f * (Gx + Gy);
  if (!(E0 > 0.f)) return false;
  const float x = 1.0f - n_r2_far / (Gx + Gy);
  if (!(x > 0.0f)) return false;  // no pair of these radii is beyond the threshold for sure
  float m[4][4], c2, c1, c0;
  qcp_coeffs(H, E0, m, c2, c1, c0);
  const float x2 = x * x;
  const float P = ((x2 + c2) * x + c1) * x + c0;
  const float dP = (4.0f * x2 + 2.0f * c2) * x + c1;
  const float d2P = 12.0f * x2 + 2.0f * c2;
  return P > 0.0f && dP > 0.0f && d2P > 0.0f;
}

// Unit quaternion (w, x, y, z) of the optimal rotation (R x ~ y) and the
// estimate G_x + G_y - 2 lambda_max (>= 0).  The eigenvector of N for
// lambda_max is the cofactor row of N - lambda I with the largest diagonal
// cofactor.  Identity for degenerate input.
__device__ __forceinline__ float qcp_quaternion(const float H[9], float Gx, float Gy, float q[4]) {
  q[0] = 1.f;
  q[1] = q[2] = q[3] = 0.f;
  const float E0 = 0.5f * (Gx + Gy);
  if (!(E0 > 0.f)) return 0.f;
  float m[4][4];
  const float lam = qcp_lambda(H, E0, m);
  float a[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) a[r][c] = m[r][c] - (r == c ? lam : 0.0f);
  const float d0 = fabsf(minor4(a, 0, 0)), d1 = fabsf(minor4(a, 1, 1));
  const float d2 = fabsf(minor4(a, 2, 2)), d3 = fabsf(minor4(a, 3, 3));
  float v[4];
  if (d0 >= d1 && d0 >= d2 && d0 >= d3) cofactor_row<0>(a, v);
  else if (d1 >= d2 && d1 >= d3) cofactor_row<1>(a, v);
  else if (d2 >= d3) cofactor_row<2>(a, v);
  else cofactor_row<3>(a, v);
  const float nv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
  if (nv > 0.0f && isfinite(nv)) {
    const float s = rsqrtf(nv);
    q[0] = v[0] * s;
    q[1] = v[1] * s;
    q[2] = v[2] * s;
    q[3] = v[3] * s;
  }
  return fmaxf((Gx + Gy) * (1.0f - lam), 0.0f);
}

// Row-major rotation matrix of a unit quaternion (w, x, y, z).
__device__ __forceinline__ void quat_to_rot(const float q[4], float R[9]) {
  const float w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = w * w + x * x - y * y - z * z;
  R[1] = 2.f * (x * y - w * z);
  R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);
  R[4] = w * w - x * x + y * y - z * z;
  R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);
  R[7] = 2.f * (y * z + w * x);
  R[8] = w * w - x * x - y * y + z * z;
}

}  // namespace kkm
