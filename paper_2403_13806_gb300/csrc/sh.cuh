// Real spherical harmonics up to degree 3 as Cartesian polynomials of a unit direction.
//
// Basis: real, orthonormal on the sphere, Condon-Shortley phase, coefficient index
// l*l + l + m with m = -l..l (the view-dependent colour of Sec. 3.2, "third-degree SH").
// Each normalisation constant is sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (times sqrt 2 for
// m != 0) folded with the integer factors of the expanded Legendre polynomial; the
// polynomials use x^2 + y^2 + z^2 = 1.
#pragma once

namespace rs {
namespace sh {

constexpr double kPi = 3.14159265358979323846;
// constexpr square root (Newton iteration in double), used only for the constants below
constexpr double csqrt_iter(double x, double cur, double prev) {
  return cur == prev ? cur : csqrt_iter(x, 0.5 * (cur + x / cur), cur);
}
constexpr double csqrt(double x) { return x > 0 ? csqrt_iter(x, x, 0.0) : 0.0; }

constexpr float Y00 = (float)(csqrt(1.0 / (4.0 * kPi)));             // 1/(2 sqrt(pi))
constexpr float Y1 = (float)(csqrt(3.0 / (4.0 * kPi)));
constexpr float Y2a = (float)(csqrt(15.0 / (4.0 * kPi)));             // xy, yz, xz
constexpr float Y2b = (float)(csqrt(5.0 / (16.0 * kPi)));             // 3z^2 - 1
constexpr float Y2c = (float)(csqrt(15.0 / (16.0 * kPi)));            // x^2 - y^2
constexpr float Y3a = (float)(csqrt(35.0 / (32.0 * kPi)));            // y(3x^2 - y^2), x(x^2 - 3y^2)
constexpr float Y3b = (float)(csqrt(105.0 / (4.0 * kPi)));            // xyz
constexpr float Y3c = (float)(csqrt(21.0 / (32.0 * kPi)));            // y(5z^2 - 1), x(5z^2 - 1)
constexpr float Y3d = (float)(csqrt(7.0 / (16.0 * kPi)));             // z(5z^2 - 3)
constexpr float Y3e = (float)(csqrt(105.0 / (16.0 * kPi)));           // z(x^2 - y^2)

// Y[0 .. (D+1)^2) for the unit direction (x, y, z).
template <int D>
__device__ __forceinline__ void basis(float x, float y, float z, float* Y) {
  Y[0] = Y00;
  if (D >= 1) {
    Y[1] = -Y1 * y;
    Y[2] = Y1 * z;
    Y[3] = -Y1 * x;
  }
  if (D >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = Y2a * x * y;
    Y[5] = -Y2a * y * z;
    Y[6] = Y2b * (3.0f * zz - 1.0f);
    Y[7] = -Y2a * x * z;
    Y[8] = Y2c * (xx - yy);
    if (D >= 3) {
      Y[9] = -Y3a * y * (3.0f * xx - yy);
      Y[10] = Y3b * x * y * z;
      Y[11] = -Y3c * y * (5.0f * zz - 1.0f);
      Y[12] = Y3d * z * (5.0f * zz - 3.0f);
      Y[13] = -Y3c * x * (5.0f * zz - 1.0f);
      Y[14] = Y3e * z * (xx - yy);
      Y[15] = -Y3a * x * (xx - 3.0f * yy);
    }
  }
}

// Gradient of sum_k w[k] Y_k(x, y, z) with respect to (x, y, z) (the polynomials above,
// differentiated as written; the caller projects out the radial part).
template <int D>
__device__ __forceinline__ void basis_grad(float x, float y, float z, const float* w, float& gx,
                                           float& gy, float& gz) {
  gx = 0.f;
  gy = 0.f;
  gz = 0.f;
  if (D >= 1) {
    gy += -Y1 * w[1];
    gz += Y1 * w[2];
    gx += -Y1 * w[3];
  }
  if (D >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    gx += Y2a * y * w[4];
    gy += Y2a * x * w[4];
    gy += -Y2a * z * w[5];
    gz += -Y2a * y * w[5];
    gz += Y2b * 6.0f * z * w[6];
    gx += -Y2a * z * w[7];
    gz += -Y2a * x * w[7];
    gx += Y2c * 2.0f * x * w[8];
    gy += -Y2c * 2.0f * y * w[8];
    if (D >= 3) {
      gx += -Y3a * 6.0f * x * y * w[9];
      gy += -Y3a * (3.0f * xx - 3.0f * yy) * w[9];
      gx += Y3b * y * z * w[10];
      gy += Y3b * x * z * w[10];
      gz += Y3b * x * y * w[10];
      gy += -Y3c * (5.0f * zz - 1.0f) * w[11];
      gz += -Y3c * 10.0f * y * z * w[11];
      gz += Y3d * (15.0f * zz - 3.0f) * w[12];
      gx += -Y3c * (5.0f * zz - 1.0f) * w[13];
      gz += -Y3c * 10.0f * x * z * w[13];
      gx += Y3e * 2.0f * x * z * w[14];
      gy += -Y3e * 2.0f * y * z * w[14];
      gz += Y3e * (xx - yy) * w[14];
      gx += -Y3a * (3.0f * xx - 3.0f * yy) * w[15];
      gy += Y3a * 6.0f * x * y * w[15];
    }
  }
}

}  // namespace sh
}  // namespace rs
