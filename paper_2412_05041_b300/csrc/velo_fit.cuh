// Track fit of the first stage (Sec. "HLT1 details and results": a
// parameterised Kalman filter over the pixel-tracker segment only), in
// binary32 with every operation rounded once in the order written here:
//  * straight-line least squares per projection, sums S0 = n, Sz, Szz, Sx,
//    Sxz (then Sy, Syz) over the hits ascending in z with dz = z - z_first;
//    det = S0 Szz - Sz^2, tx = (S0 Sxz - Sz Sx) / det, x = (Sx - tx Sz) / S0;
//    chi2 = sum over hits of (((x_i - x) - tx dz_i) / sigma)^2, both projections;
//    z_beam = z_first - (x tx + y ty) / (tx^2 + ty^2)  (z_first if tx = ty = 0);
//  * simplified Kalman filter per projection, downstream to upstream, started
//    at the second-to-last hit from the last two (no prior):
//    X = m[n-2], T = (m[n-2] - m[n-1]) / dz0, C = [[s2, s2/dz0], [s2/dz0, 2 s2/dz0^2 + q]];
//    predict F = [[1, dz], [0, 1]], Q = diag(0, q = theta^2); update H = [1, 0],
//    R = s2 = sigma^2; chi2 += r^2 / S per update.
#pragma once

#include "velo.h"

namespace velo {

__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fd(float a, float b) { return __fdiv_rn(a, b); }

__device__ __forceinline__ void kalman_1d(uint32_t n, const float* z, const float* m, float sigma, float theta,
                                          float out[5], float* chi2_out) {
  const float s2 = fm(sigma, sigma), q = fm(theta, theta);
  const float dz0 = fs(z[n - 2], z[n - 1]);
  float X = m[n - 2];
  float T = fd(fs(m[n - 2], m[n - 1]), dz0);
  float C00 = s2;
  float C01 = fd(s2, dz0);
  float C11 = fa(fd(fa(s2, s2), fm(dz0, dz0)), q);
  float chi2 = 0.0f;
  for (int i = (int)n - 3; i >= 0; --i) {
    const float dz = fs(z[i], z[i + 1]);
    X = fa(X, fm(T, dz));
    const float t1 = fm(C11, dz);
    C00 = fa(C00, fm(dz, fa(fa(C01, C01), t1)));
    C01 = fa(C01, t1);
    C11 = fa(C11, q);
    const float r = fs(m[i], X);
    const float S = fa(C00, s2);
    const float K0 = fd(C00, S), K1 = fd(C01, S);
    X = fa(X, fm(K0, r));
    T = fa(T, fm(K1, r));
    C11 = fs(C11, fm(K1, C01));
    C01 = fs(C01, fm(K0, C01));
    C00 = fs(C00, fm(K0, C00));
    chi2 = fa(chi2, fd(fm(r, r), S));
  }
  out[0] = X;
  out[1] = T;
  out[2] = C00;
  out[3] = C01;
  out[4] = C11;
  *chi2_out = chi2;
}

// Full state (VELO_STATE_STRIDE floats, layout in velo.h) of one track whose
// hits are given ascending in z.
__device__ __forceinline__ void fit_track(uint32_t n, const float* x, const float* y, const float* z, float sigma,
                                          float theta, float* st) {
  const float z0 = z[0];
  const float S0 = (float)n;
  float Sz = 0.0f, Szz = 0.0f, Sx = 0.0f, Sxz = 0.0f, Sy = 0.0f, Syz = 0.0f;
  for (uint32_t i = 0; i < n; ++i) {
    const float dz = fs(z[i], z0);
    Sz = fa(Sz, dz);
    Szz = fa(Szz, fm(dz, dz));
    Sx = fa(Sx, x[i]);
    Sxz = fa(Sxz, fm(x[i], dz));
    Sy = fa(Sy, y[i]);
    Syz = fa(Syz, fm(y[i], dz));
  }
  const float det = fs(fm(S0, Szz), fm(Sz, Sz));
  const float tx = fd(fs(fm(S0, Sxz), fm(Sz, Sx)), det);
  const float xx = fd(fs(Sx, fm(tx, Sz)), S0);
  const float ty = fd(fs(fm(S0, Syz), fm(Sz, Sy)), det);
  const float yy = fd(fs(Sy, fm(ty, Sz)), S0);
  float chi2 = 0.0f;
  for (uint32_t i = 0; i < n; ++i) {
    const float dz = fs(z[i], z0);
    const float rx = fd(fs(fs(x[i], xx), fm(tx, dz)), sigma);
    chi2 = fa(chi2, fm(rx, rx));
    const float ry = fd(fs(fs(y[i], yy), fm(ty, dz)), sigma);
    chi2 = fa(chi2, fm(ry, ry));
  }
  const float num = fa(fm(xx, tx), fm(yy, ty));
  const float den = fa(fm(tx, tx), fm(ty, ty));
  const float zb = den > 0.0f ? fs(z0, fd(num, den)) : z0;
  float kx[5], ky[5], cx2, cy2;
  kalman_1d(n, z, x, sigma, theta, kx, &cx2);
  kalman_1d(n, z, y, sigma, theta, ky, &cy2);
  st[0] = xx;
  st[1] = yy;
  st[2] = tx;
  st[3] = ty;
  st[4] = z0;
  st[5] = zb;
  st[6] = chi2;
  st[7] = fa(cx2, cy2);
  st[8] = kx[0];
  st[9] = ky[0];
  st[10] = kx[1];
  st[11] = ky[1];
  st[12] = kx[2];
  st[13] = kx[3];
  st[14] = kx[4];
  st[15] = ky[2];
  st[16] = ky[3];
  st[17] = ky[4];
  st[18] = (float)(2 * n - 4);
  st[19] = 0.0f;
}

// The plain method's keep decision: chi2/ndf <= chi2ndf_max (LSQ chi2 when
// theta == 0, Kalman chi2 otherwise), and <= chi2ndf_max_3hit for 3 hits.
__device__ __forceinline__ bool keep_track(uint32_t n, const float* st, float theta, float cut, float cut3) {
  const float chi2 = theta == 0.0f ? st[6] : st[7];
  const float r = fd(chi2, (float)(2 * n - 4));
  if (n == 3 && !(r <= cut3)) return false;
  return r <= cut;
}

}  // namespace velo
