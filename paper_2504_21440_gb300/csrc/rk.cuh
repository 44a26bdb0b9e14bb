// Embedded 7-stage FSAL Runge-Kutta 5(4) pairs and the step-size controller,
// as device constants.
//
// Dormand & Prince (1980), J. Comput. Appl. Math. 6, 19-26, and
// Tsitouras (2011), Comput. Math. Appl. 62, 770-775.  RK_E holds the error
// weights b - bhat.  Row 6 of RK_A equals b (first same as last): the last
// stage is evaluated at the new solution and reused as the next step's first.
#pragma once

#include <cuda_runtime.h>

namespace qtl {

struct RkTab {
    double c[7];
    double a[7][7];
    double e[7];
};

static __constant__ RkTab RK_TABS[2] = {
    // QTL_DP5
    {{0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0},
     {{0, 0, 0, 0, 0, 0, 0},
      {1.0 / 5.0, 0, 0, 0, 0, 0, 0},
      {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0, 0},
      {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0, 0},
      {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0, 0},
      {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0, 0},
      {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0, 0}},
     {71.0 / 57600.0, 0.0, -71.0 / 16695.0, 71.0 / 1920.0, -17253.0 / 339200.0, 22.0 / 525.0,
      -1.0 / 40.0}},
    // QTL_TSIT5
    {{0.0, 0.161, 0.327, 0.9, 0.9800255409045097, 1.0, 1.0},
     {{0, 0, 0, 0, 0, 0, 0},
      {0.161, 0, 0, 0, 0, 0, 0},
      {-0.008480655492356989, 0.335480655492357, 0, 0, 0, 0, 0},
      {2.897153057105493, -6.359448489975075, 4.3622954328695815, 0, 0, 0, 0},
      {5.325864828439257, -11.748883564062828, 7.4955393428898365, -0.09249506636175525, 0, 0, 0},
      {5.86145544294642, -12.92096931784711, 8.159367898576159, -0.071584973281401,
       -0.028269050394068383, 0, 0},
      {0.09646076681806523, 0.01, 0.4798896504144996, 1.379008574103742, -3.290069515436081,
       2.324710524099774, 0}},
     {-0.00178001105222577714, -0.0008164344596567469, 0.007880878010261995,
      -0.1447110071732629, 0.5823571654525552, -0.45808210592918697, 0.015151515151515152}},
};

// PI controller (readings of the integrator the paper leaves to its ODE
// library): accept fac = 0.9 err^-0.14 err_prev^0.08 in [0.2, 10], at most 1
// right after a reject, err_prev floored at 1e-4; reject fac = max(0.2, 0.9 err^-0.2).
struct Controller {
    double err_prev;
    bool last_rejected;

    __device__ void init() {
        err_prev = 1e-4;
        last_rejected = false;
    }
    __device__ double on_accept(double err) {
        double fac;
        if (err == 0.0)
            fac = 10.0;
        else
            fac = 0.9 * pow(err, -0.7 / 5.0) * pow(err_prev, 0.4 / 5.0);
        fac = fmin(10.0, fmax(0.2, fac));
        if (last_rejected) fac = fmin(fac, 1.0);
        err_prev = fmax(err, 1e-4);
        last_rejected = false;
        return fac;
    }
    __device__ double on_reject(double err) {
        last_rejected = true;
        return fmax(0.2, 0.9 * pow(err, -1.0 / 5.0));
    }
};

// The same factors evaluated in FP32 by a single thread (GB300's FP64 pipe is
// 1/64 rate; the factor only steers the step size, so its last bits do not
// matter -- the FP64 oracle's results move by < 3e-13 when its factor is
// rounded to FP32).
struct CtlF {
    float err_prev;
    bool last_rejected;
    __device__ void init() {
        err_prev = 1e-4f;
        last_rejected = false;
    }
    __device__ float on_accept(float err) {
        float fac = err == 0.0f ? 10.0f
                                : 0.9f * exp2f(-0.14f * log2f(err) + 0.08f * log2f(err_prev));
        fac = fminf(10.0f, fmaxf(0.2f, fac));
        if (last_rejected) fac = fminf(fac, 1.0f);
        err_prev = fmaxf(err, 1e-4f);
        last_rejected = false;
        return fac;
    }
    __device__ float on_reject(float err) {
        last_rejected = true;
        return fmaxf(0.2f, 0.9f * exp2f(-0.2f * log2f(err)));
    }
};

// A step lands on the next output time when it falls short of it by at most
// 64 units of 2^-52 max(1, |t_target|).
__device__ __forceinline__ bool lands(double h, double t, double t_target) {
    return h >= (t_target - t) - 64.0 * 0x1p-52 * fmax(1.0, fabs(t_target));
}

// The step to try toward the next output time t_target from t, with the
// controller's step h: the rest of the way when h lands on it; with adaptive
// steps, half the rest when h covers more than half of it, so that two equal
// steps land instead of a full step and a short remainder (whose small size
// the controller would then have to grow back); else h.
__device__ __forceinline__ double step_toward(double h, double t, double t_target, bool fixed, bool* land) {
    const double rem = t_target - t;
    *land = lands(h, t, t_target);
    if (*land) return rem;
    if (!fixed && h >= 0.5 * rem) return 0.5 * rem;
    return h;
}

// Starting step of Hairer, Norsett & Wanner (Solving ODEs I, Sec. II.4) for a
// method of order 5, from the RMS norms d0 = |y0|, d1 = |f0|, d2 = |f1-f0|/h0.
__device__ __forceinline__ double start_h0(double d0, double d1) {
    return (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
}
__device__ __forceinline__ double start_h(double h0, double d1, double d2) {
    double m = fmax(d1, d2);
    double h1 = (m <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / m, 1.0 / 5.0);
    return fmin(100.0 * h0, h1);
}

}  // namespace qtl
