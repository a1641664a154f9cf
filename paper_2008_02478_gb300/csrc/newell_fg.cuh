// Newell's auxiliary functions f and g (Table 1: demagnetising tensor from
// Newell, Williams and Dunlop, Ref. [50] of the paper), shared by the single-
// and multi-mesh tensor builders.
#pragma once
#include <cuda_runtime.h>

namespace boris {

// Newell's f: even in each argument; a term with a vanishing polynomial factor
// is dropped (its closed-form limit is zero).
__device__ __forceinline__ double newell_f_dev(double x, double y, double z)
{
    x = fabs(x); y = fabs(y); z = fabs(z);
    const double xx = x * x, yy = y * y, zz = z * z;
    const double R = sqrt(xx + yy + zz);
    if (R == 0.0) return 0.0;
    double acc = (2.0 * xx - yy - zz) * R * (1.0 / 6.0);
    const double t1 = 0.5 * y * (zz - xx);
    if (t1 != 0.0) acc += t1 * asinh(y / sqrt(xx + zz));
    const double t2 = 0.5 * z * (yy - xx);
    if (t2 != 0.0) acc += t2 * asinh(z / sqrt(xx + yy));
    const double t3 = x * y * z;
    if (t3 != 0.0) acc -= t3 * atan(y * z / (x * R));
    return acc;
}

// Newell's g: odd in x and y, even in z.
__device__ __forceinline__ double newell_g_dev(double x, double y, double z)
{
    const double sign = copysign(1.0, x) * copysign(1.0, y);
    x = fabs(x); y = fabs(y); z = fabs(z);
    const double xx = x * x, yy = y * y, zz = z * z;
    const double R = sqrt(xx + yy + zz);
    if (R == 0.0) return 0.0;
    double acc = -x * y * R * (1.0 / 3.0);
    const double xyz = x * y * z;
    if (xyz != 0.0) acc += xyz * asinh(z / sqrt(xx + yy));
    const double a = y * (3.0 * zz - yy) * (1.0 / 6.0);
    if (a != 0.0) acc += a * asinh(x / sqrt(yy + zz));
    const double b = x * (3.0 * zz - xx) * (1.0 / 6.0);
    if (b != 0.0) acc += b * asinh(y / sqrt(xx + zz));
    if (z != 0.0) {
        acc -= zz * z * (1.0 / 6.0) * atan(x * y / (z * R));
        if (y != 0.0) acc -= 0.5 * z * yy * atan(x * z / (y * R));
        if (x != 0.0) acc -= 0.5 * z * xx * atan(y * z / (x * R));
    }
    return sign * acc;
}

}  // namespace boris
