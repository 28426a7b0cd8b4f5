// Real spherical harmonics up to degree 3 as Cartesian polynomials of a unit
// direction (x, y, z), for the per-point colour of Sec. 3.1 Eq. 4.
//
// Convention: real orthonormal SH without the Condon-Shortley phase, index
// k = l*l + l + m.  The constants are the normalisations
// sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (times sqrt 2 for m != 0) multiplied
// into the polynomial form of each function.
#pragma once

namespace pbr {

namespace shc {
constexpr float C0 = 0.28209479177387814f;
constexpr float C1 = 0.4886025119029199f;
constexpr float C2a = 1.0925484305920792f;  // xy, yz, xz
constexpr float C2b = 0.31539156525252005f; // 3z^2 - 1
constexpr float C2c = 0.5462742152960396f;  // x^2 - y^2
constexpr float C3a = 0.5900435899266435f;  // y(3x^2-y^2), x(x^2-3y^2)
constexpr float C3b = 2.890611442640554f;   // xyz
constexpr float C3c = 0.4570457994644658f;  // y(5z^2-1), x(5z^2-1)
constexpr float C3d = 0.3731763325901154f;  // z(5z^2-3)
constexpr float C3e = 1.445305721320277f;   // z(x^2-y^2)
} // namespace shc

template <int DEG> struct SH {
    static constexpr int K = (DEG + 1) * (DEG + 1);
};

// Y[k] at the unit direction (x, y, z).
template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y)
{
    using namespace shc;
    Y[0] = C0;
    if (DEG >= 1) {
        Y[1] = C1 * y;
        Y[2] = C1 * z;
        Y[3] = C1 * x;
    }
    if (DEG >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = C2a * x * y;
        Y[5] = C2a * y * z;
        Y[6] = C2b * (3.0f * zz - 1.0f);
        Y[7] = C2a * x * z;
        Y[8] = C2c * (xx - yy);
        if (DEG >= 3) {
            Y[9] = C3a * y * (3.0f * xx - yy);
            Y[10] = C3b * x * y * z;
            Y[11] = C3c * y * (5.0f * zz - 1.0f);
            Y[12] = C3d * z * (5.0f * zz - 3.0f);
            Y[13] = C3c * x * (5.0f * zz - 1.0f);
            Y[14] = C3e * z * (xx - yy);
            Y[15] = C3a * x * (xx - 3.0f * yy);
        }
    }
}

// g += sum_k w[k] * grad Y_k(x, y, z)  (Cartesian gradient of the polynomial
// form; the caller projects it onto the tangent plane of the unit sphere).
template <int DEG>
__device__ __forceinline__ void sh_grad_accum(float x, float y, float z, const float *w,
                                              float &gx, float &gy, float &gz)
{
    using namespace shc;
    if (DEG >= 1) {
        gy += C1 * w[1];
        gz += C1 * w[2];
        gx += C1 * w[3];
    }
    if (DEG >= 2) {
        gx += C2a * (y * w[4] + z * w[7]) + 2.0f * C2c * x * w[8];
        gy += C2a * (x * w[4] + z * w[5]) - 2.0f * C2c * y * w[8];
        gz += C2a * (y * w[5] + x * w[7]) + 6.0f * C2b * z * w[6];
        if (DEG >= 3) {
            const float xx = x * x, yy = y * y, zz = z * z;
            gx += C3a * 6.0f * x * y * w[9] + C3b * y * z * w[10] + C3c * (5.0f * zz - 1.0f) * w[13] +
                  C3e * 2.0f * x * z * w[14] + C3a * 3.0f * (xx - yy) * w[15];
            gy += C3a * 3.0f * (xx - yy) * w[9] + C3b * x * z * w[10] + C3c * (5.0f * zz - 1.0f) * w[11] -
                  C3e * 2.0f * y * z * w[14] - C3a * 6.0f * x * y * w[15];
            gz += C3b * x * y * w[10] + C3c * 10.0f * y * z * w[11] + C3d * (15.0f * zz - 3.0f) * w[12] +
                  C3c * 10.0f * x * z * w[13] + C3e * (xx - yy) * w[14];
        }
    }
}

} // namespace pbr
