// Initial conditions at a point (the mesh kernels of geometry.cu and
// aniso.cu): the isentropic vortex (Shu) advected by the free stream for a
// time ic.t, periodic in x and y, and the Taylor-Green vortex.
#pragma once

#include <math.h>

#include "hs3d.h"

namespace hs3d {

__device__ __forceinline__ void ic_point(const hs3d_ic &ic, double Lx, double Ly, double x, double y, double z,
                                         double u[5])
{
    double g = ic.gamma;
    double rho, v1, v2, v3, pr;
    if (ic.kind == HS3D_IC_VORTEX) {
        double uinf = ic.Ma * sqrt(g);
        double dx = x - (ic.xc + uinf * ic.t), dy = y - ic.yc;
        dx -= Lx * floor(dx / Lx + 0.5);
        dy -= Ly * floor(dy / Ly + 0.5);
        double r2 = dx * dx + dy * dy;
        double ex = exp(0.5 * (1.0 - r2));
        double k = ic.beta / (2.0 * M_PI);
        v1 = uinf - k * ex * dy;
        v2 = k * ex * dx;
        v3 = 0.0;
        double T = 1.0 - (g - 1.0) * ic.beta * ic.beta / (8.0 * g * M_PI * M_PI) * ex * ex;
        rho = pow(T, 1.0 / (g - 1.0));
        pr = rho * T;
    } else {
        double p0 = 1.0 / (g * ic.Ma * ic.Ma);
        v1 = sin(x) * cos(y) * cos(z);
        v2 = -cos(x) * sin(y) * cos(z);
        v3 = 0.0;
        pr = p0 + (cos(2.0 * x) + cos(2.0 * y)) * (cos(2.0 * z) + 2.0) * (1.0 / 16.0);
        rho = pr / p0;
    }
    u[0] = rho;
    u[1] = rho * v1;
    u[2] = rho * v2;
    u[3] = rho * v3;
    u[4] = pr / (g - 1.0) + 0.5 * rho * (v1 * v1 + v2 * v2 + v3 * v3);
}

}  // namespace hs3d
