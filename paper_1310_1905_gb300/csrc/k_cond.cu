// Condensation / evaporation (paper Sec. 5.1.3): a group of lanes per grid
// cell, all sstp_cond substeps in one launch.  In each substep every lane
// advances its super-droplets' r_w^2 with the implicit growth equation (eq.
// rw2_implicit), the group sums N (r_w^3[new] - r_w^3[old]) and every lane
// applies eq. (rhov_update) to its register copy of the cell's r_v, theta.
#include "sdm_internal.cuh"

namespace sdm {

SDM_HD double fres(double x, double x0, double rd3, double kappa,
                                       const Thermo &t, double dtp, int physics) {
    return x - x0 - dtp * growth(x, rd3, kappa, t, physics);
}

// The paper's predictor-corrector: bracket [a, b] from the derivative at
// x0 with the factor 2, the Euler step (a+b)/2 when f does not change strict
// sign over it, bisection to b - a <= 2^-52 b otherwise.
__host__ __device__ double solve_rw2_bisect(double x0, double rd3, double kappa, const Thermo &t,
                                   double dtp, int physics, int *euler) {
    const double g0 = growth(x0, rd3, kappa, t, physics);
    const double a = fmax(rd2_of(rd3), x0 + fmin(2.0 * dtp * g0, 0.0));
    const double b = x0 + fmax(2.0 * dtp * g0, 0.0);
    const double fa = fres(a, x0, rd3, kappa, t, dtp, physics);
    const double fb = fres(b, x0, rd3, kappa, t, dtp, physics);
    if ((fa > 0.0) == (fb > 0.0)) {
        *euler = 1;
        return 0.5 * (a + b);
    }
    double lo = a, hi = b;
    const bool plo = fa > 0.0;
    for (int it = 0; it < 200; ++it) {
        if (hi - lo <= 0x1p-52 * hi) break;
        const double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        const bool pm = fres(mid, x0, rd3, kappa, t, dtp, physics) > 0.0;
        if (pm == plo) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// ---------------------------------------------------------------------------
// Fast solve, faithful to the bisection.  The bracket and the ill-posedness
// test are those of solve_rw2_bisect (FP64).  The sign of f at a point is
// first computed in FP32 with an error bound and trusted where |f| exceeds
// it.  (1) The bisection runs on the FP32 increment d = x - x0 while FP32
// decides; (2) where it stops deciding, a bracketed Newton/secant iteration
// in FP64 converges to a sign change inside the bracket; (3) an FP32 replay
// of the remaining halvings checks that the bisection leads to that same
// sign change (near activation there can be several).  If the iteration
// does not settle or the replay leaves its root, the exact FP64 bisection
// finishes the job.
struct ThermoF {
    float rho_vs, rho_v_eff, A, Dterm, lambda_D, lambda_K, Sc, Pr, cX;
};

SDM_HD ThermoF to_float(const Thermo &t) {
    ThermoF f;
    f.rho_vs = (float)t.rho_vs;
    f.rho_v_eff = (float)t.rho_v_eff;
    f.A = (float)t.A;
    f.Dterm = (float)t.Dterm;
    f.lambda_D = (float)t.lambda_D;
    f.lambda_K = (float)t.lambda_K;
    f.Sc = (float)t.Sc;
    f.Pr = (float)t.Pr;
    f.cX = (float)t.cX;
    return f;
}

// a / b within 2 ulps (the device's fast division; exact on the host).  The
// FP32 growth rate below uses it throughout: its error bound allows 16 ulps
// of rho_o, 8 amp of a_w and 64 of the D_eff factor, so 2-ulp quotients stay
// well inside it, and the fast form keeps the kernels' code small.
SDM_HD float fdiv(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
}

SDM_HD float fs_f(float Kn) {
    return fdiv(1.0f + Kn, 1.0f + (4.0f / 3.0f + 0.377f) * Kn + 4.0f / 3.0f * Kn * Kn);
}

// FP32 growth rate g and an absolute error bound for it; with DG > 0 also
// its derivative dg/dx: DG = 1 through the Koehler factor only, DG = 2 also
// through D_eff's variation with r (transition regime and ventilation), for
// the polish's first Newton step.
enum { kDgNone = 0, kDgKoehler = 1, kDgFull = 2 };

template <int DG>
SDM_HD float growth_f(float x, float rd3, float kappa, const ThermoF &t, int physics, float *err, float *dgdx,
                      float *edg = nullptr, float *curv = nullptr, float *mag = nullptr) {
    const float r = sqrtf(x);
    const float r3 = x * r;
    const float num = r3 - rd3, den = r3 - rd3 * (1.0f - kappa);
    const float aw = fdiv(num, den);
    const float Ar = fdiv(t.A, r);
    const float kel = expf(Ar);
    const float rho_o = t.rho_vs * aw * kel;
    float D = (float)phys::D0, K = (float)phys::K0;
    float dlnD = 0.0f, dlnK = 0.0f;  // d ln D / d ln r, d ln K / d ln r
    if (physics) {
        const float c1 = 4.0f / 3.0f + 0.377f, c2 = 4.0f / 3.0f;
        const float KnM = fdiv(t.lambda_D, r), KnT = fdiv(t.lambda_K, r);
        const float bM = fs_f(KnM), bT = fs_f(KnT);
        const float X = t.cX * r3;
        const float ce = (float)(4.0 / (phys::delta0 * phys::delta0 * 0.54037024344425184));  // sqrt(C0)
        const float e = ce * sqrtf(X);
        const float sq = sqrtf(1.0f + e);
        const float s = fdiv(e, sq + 1.0f);
        const float Re = (float)(phys::delta0 * phys::delta0 / 4.0) * s * s;
        const float fRe = Re > 1.0f ? powf(Re, 0.077f) : 1.0f;
        const float qS = cbrtf(1.0f + Re * t.Sc), qP = cbrtf(1.0f + Re * t.Pr);
        const float Sh = 1.0f + qS * fRe, Nu = 1.0f + qP * fRe;
        D = (float)phys::D0 * bM * Sh * 0.5f;
        K = (float)phys::K0 * bT * Nu * 0.5f;
        if (DG == kDgFull) {
            // d ln beta / d ln r = -d ln beta / d ln Kn
            auto dlnbeta = [&](float Kn) {
                return (c1 * Kn + 2.0f * c2 * Kn * Kn) / (1.0f + c1 * Kn + c2 * Kn * Kn) - Kn / (1.0f + Kn);
            };
            // Re(X), X ~ r^3: d ln Re / d ln r = 3 e / (2 s sqrt(1 + e))
            const float dlnRe = s > 0.0f ? 3.0f * e / (2.0f * s * sq) : 3.0f;
            const float dfRe = Re > 1.0f ? 0.077f : 0.0f;  // d ln fRe / d ln Re
            const float dSh = fRe * (Re * t.Sc / (3.0f * qS * qS) + dfRe * qS) * dlnRe / Sh;
            const float dNu = fRe * (Re * t.Pr / (3.0f * qP * qP) + dfRe * qP) * dlnRe / Nu;
            dlnD = dlnbeta(KnM) + dSh;
            dlnK = dlnbeta(KnT) + dNu;
        }
    }
    const float Deff = fdiv(1.0f, fdiv(1.0f, D) + fdiv(t.Dterm, K));
    const float c = 2.0f * Deff / (float)phys::rho_w;
    const float g = c * (t.rho_v_eff - rho_o);
    // Error bound.  u = 2^-24; a correctly rounded FP32 operation or
    // conversion errs by at most u (relative), the 2-ulp division fdiv by
    // 4u, expf (2 ulps) by 4u, sqrtf (correctly rounded) by u, cbrtf (1 ulp)
    // by 2u, powf (4 ulps) by 8u; to first order, relative errors add along
    // a chain and scale by the logarithmic sensitivity of the result.
    // - The point x = x0f + d errs by 2u (x0's conversion, the sum), r3 by
    //   5u (x^1.5, the root, the product).
    // - rho_v_eff: one conversion, u.
    // - rho_o = rho_vs a_w e^(A/r): a_w = num/den moves with r3 by at most
    //   kappa r3 rd3 / (num den) <= amp per unit relative change of r3 (num
    //   and den move together), so 5u amp; the roundings of rd3 and of the
    //   two differences, u (r3 + rd3)/|num| <= u amp and 2u; fdiv 4u: a_w
    //   within (6 amp + 6) u.  A/r: A's conversion, the root, fdiv: 7u, so
    //   e^(A/r) within 7u A/r + 4u.  rho_vs and two products: 3u.  In all
    //   (13 + 6 amp + 7 A/r) u, inside the (16 + 8 amp + 8 A/r) u taken.
    // - the factor c = 2 D_eff / rho_w: through X, e, s and Re (23u), the
    //   cube roots (11u each), Re^0.077 (10u), Kn and the transition factors
    //   (15u each), D and K (41u), D_eff (51u) and c (53u), inside the 64u
    //   of |g| taken for it.
    // The sign of f = d - dt' g taken from this value is then the one an
    // FP64 evaluation at x0 + d gives wherever |f| clears the callers'
    // margin (4u |d| for the rounding of d and of the difference, plus
    // 4 dt' err).
    const float amp = fdiv(r3 + rd3, fmaxf(fabsf(num), 1e-37f));
    const float eps = 5.9604645e-8f;  // 2^-24
    *err = eps * (c * (4.0f * t.rho_v_eff + rho_o * (16.0f + 8.0f * amp + 8.0f * Ar)) + 64.0f * fabsf(g));
    if (DG != kDgNone) {
        // 3 r^2 rd3 kappa / den^2 without squaring den (~1e-24 m^3 for 10 nm
        // droplets, whose square underflows FP32)
        const float drho_dr = t.rho_vs * kel * (3.0f * kappa * fdiv(rd3, den) * fdiv(x, den) - aw * fdiv(t.A, x));
        // D_eff = 1 / (1/D + Dterm/K): d ln D_eff = (D_eff/D) d ln D + (1 - D_eff/D) d ln K
        const float wD = Deff / D;
        const float dlnc = wD * dlnD + (1.0f - wD) * dlnK;
        *dgdx = (g * dlnc - c * drho_dr * r) / (2.0f * x);
        if (DG == kDgFull && edg) {
            // an absolute bound of dg/dx's error: g carries err; the Koehler
            // slope's two terms, D_eff's logarithmic derivatives and the
            // factor c each carry a few tens of FP32 ulps (2^-16 covers them
            // with room)
            const float mk = t.rho_vs * kel * (3.0f * kappa * fdiv(rd3, den) * fdiv(x, den) + aw * fdiv(t.A, x));
            *edg = (*err * fabsf(dlnc) +
                    1.52587890625e-5f * (fabsf(g) * (fabsf(dlnc) + fabsf(dlnD) + fabsf(dlnK) + 1.0f) + c * mk * r)) /
                   (2.0f * x);
            // x^2 |g''| bounded from the scales on which the Koehler factor
            // varies: ln a_w by up to 1.5 amp, the Kelvin factor by A/r, the
            // D_eff factor by O(1), per unit ln x
            const float sc = 2.0f + 1.5f * amp + Ar;
            *curv = c * (2.0f * fabsf(t.rho_v_eff - rho_o) + rho_o * sc * sc) / (x * x);
            *mag = c * (t.rho_v_eff + rho_o);  // the size of the terms whose difference g is
        }
    }
    return g;
}

struct SolveCounters {
    int euler, fallback;
    int evals;      // FP64 growth evaluations of the fast solve: the cost measure of the launch order
    int certified;  // solves settled by a certified Newton step (staged layout)
};

// The growth rate of eq. (maxmason) rearranged for FP64 throughput: with
// r^-1 computed once, Kn = lambda r^-1, and beta = (1 + Kn)/D(Kn),
//   D = a / D_M, K = b / D_T,   a = D0 (1 + Kn_M) Sh/2,  b = K0 (1 + Kn_T) Nu/2,
//   D_eff = D K / (K + Dterm D) = a b / (b D_M + Dterm a D_T),
//   a_w = num / den,
// so that g = 2 a b (rho_v den - rho_vs num e^(A/r)) / (rho_w (b D_M + Dterm a D_T) den)
// takes one division where the term-by-term form takes about ten.  It equals
// growth() up to rounding.  Coef holds the factor 2 D_eff / rho_w as the
// fraction (2 a b) / (rho_w (b D_M + Dterm a D_T)), numerator and denominator
// apart.
struct Coef {
    double n, d;
};

// (1 + y)^(1/3) - 1 for 0 <= y <= 1/64 by its binomial series to y^8
// (remainder below 5e-17 y, i.e. 2e-19 of Sh): the growth rate's ventilation
// factors take it for small droplets, where cbrt(1 + y) would spend an FP64
// cube root on a number within 2% of one
SDM_HD double cbrt1p_small(double y) {
    return y * (1.0 / 3 + y * (-1.0 / 9 + y * (5.0 / 81 + y * (-10.0 / 243 + y * (22.0 / 729 +
           y * (-154.0 / 6561 + y * (374.0 / 19683 + y * (-935.0 / 59049))))))));
}

// sqrt(1 + e) - 1 for 0 <= e <= 1/64 by its binomial series to e^9
// (remainder below 6e-19 e)
SDM_HD double sqrt1pm1_small(double e) {
    return e * (0.5 + e * (-1.0 / 8 + e * (1.0 / 16 + e * (-5.0 / 128 + e * (7.0 / 256 + e * (-21.0 / 1024 +
           e * (33.0 / 2048 + e * (-429.0 / 32768 + e * (715.0 / 65536)))))))));
}

// LITE: where the ventilation corrections Sh - 2 and Nu - 2 (about Re Sc/3
// and Re Pr/3) are below 2^-24 - the haze and small cloud droplets - they
// are taken in FP32: with a relative error below 2^-20 each (the chain of a
// few correctly rounded FP32 operations) they move the coefficient by less
// than 2^-45 of itself, which moves the root of the implicit equation by
// less than 2^-45 of its increment x1 - x0.  The staged solves take it; the
// fused kernel's and the bisection's coefficient stays FP64 throughout.
template <bool LITE = false>
SDM_HD Coef growth_coef(double rinv, double r3, const Thermo &t, int physics, const ThermoF *tf = nullptr) {
    using namespace phys;
    double a = D0, b = K0, DM = 1.0, DT = 1.0;
    if (physics) {
        const double c1 = 4.0 / 3.0 + 0.377, c2 = 4.0 / 3.0;
        const double KnM = t.lambda_D * rinv, KnT = t.lambda_K * rinv;
        DM = 1.0 + c1 * KnM + c2 * KnM * KnM;
        DT = 1.0 + c1 * KnT + c2 * KnT * KnT;
        if (LITE) {
            // tf: the FP32 copies of cX, Sc and Pr (the same roundings as (float) here)
            const float cXf = tf ? tf->cX : (float)t.cX, Scf = tf ? tf->Sc : (float)t.Sc;
            const float Prf = tf ? tf->Pr : (float)t.Pr;
            const float Xf = cXf * (float)r3;
            const float ef = (float)(4.0 / (delta0 * delta0 * sqrt(C0))) * sqrtf(Xf);
            const float sf = ef / (sqrtf(1.0f + ef) + 1.0f);
            const float Ref = (float)(delta0 * delta0 / 4.0) * sf * sf;
            const float yS = Ref * Scf, yN = Ref * Prf;
            if (fmaxf(yS, yN) <= 5.9604645e-8f) {  // 2^-24: (1 + y)^(1/3) - 1 = y/3 - y^2/9 + ...
                const double Sh = 2.0 + (double)(yS * (0.33333333f - 0.11111111f * yS));
                const double Nu = 2.0 + (double)(yN * (0.33333333f - 0.11111111f * yN));
                a = D0 * (1.0 + KnM) * Sh * 0.5;
                b = K0 * (1.0 + KnT) * Nu * 0.5;
                return Coef{2.0 * a * b, rho_w * (b * DM + t.Dterm * a * DT)};
            }
        }
        const double X = t.cX * r3;
        const double e = 4.0 / (delta0 * delta0 * sqrt(C0)) * sqrt(X);
        // Re = delta0^2/4 (sqrt(1 + e) - 1)^2 (KC2002)
        const double s = e <= 0.015625 ? sqrt1pm1_small(e) : e / (sqrt(1.0 + e) + 1.0);
        const double Re = delta0 * delta0 / 4.0 * s * s;
        double Sh, Nu;
        if (Re * fmax(t.Sc, t.Pr) <= 0.015625) {
            Sh = 2.0 + cbrt1p_small(Re * t.Sc);
            Nu = 2.0 + cbrt1p_small(Re * t.Pr);
        } else {
            const double fRe = Re > 1.0 ? pow(Re, 0.077) : 1.0;
            Sh = 1.0 + cbrt(1.0 + Re * t.Sc) * fRe;
            Nu = 1.0 + cbrt(1.0 + Re * t.Pr) * fRe;
        }
        a = D0 * (1.0 + KnM) * Sh * 0.5;
        b = K0 * (1.0 + KnT) * Nu * 0.5;
    }
    return Coef{2.0 * a * b, rho_w * (b * DM + t.Dterm * a * DT)};
}

// The FP32 growth rate with its error bound and dg/dx; with BOUNDS also
// dg/dx's error bound edg, a bound curv of |d2g/dx2| and the size mag of the
// terms whose difference g is.
struct GF {
    float g, err, dg, edg, curv, mag;
};

template <int DG, bool BOUNDS = false>
SDM_HD GF growth_f3(float x, float rd3, float kappa, const ThermoF &t, int physics) {
    GF r;
    r.dg = r.edg = r.curv = r.mag = 0.0f;
    if (BOUNDS) r.g = growth_f<DG>(x, rd3, kappa, t, physics, &r.err, &r.dg, &r.edg, &r.curv, &r.mag);
    else r.g = growth_f<DG>(x, rd3, kappa, t, physics, &r.err, &r.dg);
    return r;
}

// Out-of-line copies of the FP32 growth rate keep the kernels' hot code
// small (their main stall is instruction fetch): one copy serves the locate
// loop and the replay.  The ambient state is passed by address (it lives in
// shared memory in the kernels).
SDM_HD __noinline__ GF growth_f3_call(float x, float rd3, float kappa, const ThermoF *t, int physics) {
    return growth_f3<kDgNone>(x, rd3, kappa, *t, physics);
}

SDM_HD __noinline__ GF growth_f3_full(float x, float rd3, float kappa, const ThermoF *t, int physics) {
    return growth_f3<kDgFull>(x, rd3, kappa, *t, physics);
}

SDM_HD __noinline__ GF growth_f3_bounds(float x, float rd3, float kappa, const ThermoF *t, int physics) {
    return growth_f3<kDgFull, true>(x, rd3, kappa, *t, physics);
}

// the full FP32 growth rate, with the slope's bounds for a certified solve
template <bool CERT>
SDM_HD GF growth_f3_slope(float x, float rd3, float kappa, const ThermoF *t, int physics) {
    return CERT ? growth_f3_bounds(x, rd3, kappa, t, physics) : growth_f3_full(x, rd3, kappa, t, physics);
}

// the FP64 residual with the term-by-term growth rate, on the rare paths
// (undecided bracket ends, replay decisions, the bisection fallback)
SDM_HD __noinline__ double fres_rare(double x, double x0, double rd3, double kappa, const Thermo *t,
                                     double dtp, int physics) {
    return fres(x, x0, rd3, kappa, *t, dtp, physics);
}

// The fast solve's state between its FP64 growth evaluations (g(x0) first,
// then one per polish step); solve_rw2_fast drives it.
struct FastSolve {
    double x0, rd3, kappa;
    double a, b, lo, hi, xk, xp, fp, slope, sdx, sdf, x1;
    double rd2;  // r_d^2 when the bracket's lower end is clamped to it
    double es, cv, xsp;  // certified solves: the FP32 slope's error bound, a bound of |f''|, its point
    float Lu, Hu, mu;
    int k;
    bool plo, undecided, mu_inside, pmu, have_slope, clamp;
    bool mono;  // certified solves: f proven strictly monotone on the bracket (one root: no replay)
    // deferred bracket ends (staged layout): the ends whose sign needs the
    // term-by-term FP64 residual (bits 0, 1 for a, b) and the decided signs
    uint8_t pend;
    bool pe0, pe1;
};

// 1/y from the FP32 reciprocal (within 2^-23) refined by two Newton
// iterations (error squared each time, to FP64 rounding); the FP32 range is
// checked, with the division outside it
SDM_HD double rcp_refined(double y) {
    const double ay = fabs(y);
    if (!(ay > 1e-36 && ay < 1e36)) return 1.0 / y;
    double r = (double)(1.0f / (float)y);
    r = fma(r, fma(-y, r, 1.0), r);
    return fma(r, fma(-y, r, 1.0), r);
}

// The growth rate for the fast solve, one evaluation for both of its uses
// so that the solve has one copy of it.
// exact = true: g(x0) for the bracket and the Euler step.  rho_v - rho_o,
//   where all the cancellation is, takes the operations of growth() one by
//   one; the factor 2 D_eff / rho_w, which only scales it, comes from
//   growth_coef (it differs from growth()'s by rounding, a relative 1e-16 of
//   g, which moves the Euler step by a relative 1e-16 of its increment).
// exact = false: the one-division form above (the polish), and in *mag the
//   same factor times rho_v + rho_o, the size of the terms whose difference
//   g is (its rounding error is a few ulps of this).
// LITE (the staged solves): the coefficient's ventilation factors in FP32
//   where they are within 2^-24 of 2 (growth_coef); r and A/r from the
//   reciprocal square root in both forms; the Kelvin factor e^(A/r) by its
//   Taylor series where A/r <= 1/32.  Each changes g by a few ulps of its
//   terms, the rounding level the certified steps already allow for.
template <bool LITE = false>
SDM_HD double growth_eval(double x, bool exact, double rd3, double kappa, const Thermo &t, int physics,
                          double *mag, const ThermoF *tf = nullptr) {
    double r, rinv;
    if (exact && !LITE) {
        r = sqrt(x);
        rinv = 1.0 / r;
    } else {
        rinv = rsqrt_hd(x);
        r = x * rinv;
    }
    const double r3 = x * r;
    const double y = exact && !LITE ? t.A / r : t.A * rinv;
    double kel;
    if (LITE && y <= 0.03125) {
        // e^y by its Taylor series to y^8: the remainder is below
        // y^9/9! e^y < 2e-19 for y <= 1/32 (droplets above about 40 nm)
        kel = 1.0 + y * (1.0 + y * (1.0 / 2 + y * (1.0 / 6 + y * (1.0 / 24 + y * (1.0 / 120 + y * (1.0 / 720 +
              y * (1.0 / 5040 + y * (1.0 / 40320))))))));
    } else {
        kel = exp(y);
    }
    const Coef c = growth_coef<LITE>(rinv, r3, t, physics, tf);
    const double num = r3 - rd3, den = r3 - rd3 * (1.0 - kappa);
    if (exact) {
        *mag = 0.0;
        return c.n / c.d * (t.rho_v_eff - t.rho_vs * (num / den) * kel);
    }
    // LITE: 1/(c.d den) from the FP32 reciprocal and two FP64 Newton
    // iterations (within an ulp or two of the quotient, inside the 16 ulps
    // of the terms that the polish's certificate allows for g's rounding)
    const double q = LITE ? c.n * rcp_refined(c.d * den) : c.n / (c.d * den);
    const double v = t.rho_v_eff * den, o = t.rho_vs * num * kel;
    *mag = q * (v + fabs(o));
    return q * (v - o);
}

// the exact bisection from [lo, hi] (FP64 signs, as the paper's bisection
// takes them): for a polish that does not settle or a replay that leaves r
SDM_HD __noinline__ double bisect_rest(double lo, double hi, bool plo, double x0, double rd3, double kappa,
                                       const Thermo &t, double dtp, int physics) {
    for (int it = 0; it < 200; ++it) {
        if (hi - lo <= 0x1p-52 * hi) break;
        const double m = 0.5 * (lo + hi);
        if (!(m > lo && m < hi)) break;
        if ((fres_rare(m, x0, rd3, kappa, &t, dtp, physics) > 0.0) == plo) lo = m;
        else hi = m;
    }
    return 0.5 * (lo + hi);
}

// After g0 = g(x0): bracket, ends, Euler step, locate.  Returns true when
// the solve is finished (S.x1 set); otherwise S.xk is the first polish point.
// 1. locate: from the bracket [x0 + L, x0 + H] (FP32 increments) whose ends
//    have the signs plo and !plo, halve in FP32 while FP32 decides - the
//    halves the FP64 bisection takes, up to FP32 rounding of the midpoints -
//    and set up the polish at the point mu where it stops deciding.  CERT:
//    also the bounds a certified Newton step needs (newton_certified).
template <bool CERT>
SDM_HD void fs_locate(FastSolve &S, float L, float H, bool plo, const ThermoF &tf, double dtp, int physics) {
    const double x0 = S.x0;
    const float rd3f = (float)S.rd3, kf = (float)S.kappa, dtpf = (float)dtp, x0f = (float)x0;
    float mu = 0.0f;
    bool undecided = false;
    bool mono = false;
    GF q;  // CERT, mono: the FP32 growth rate and its bounds at the last Newton point
    if (CERT && H - L <= 0.0625f * x0f) {
        // f' = 1 - dt' g' lies within dt' (edg + curv |x - xm|) of the FP32
        // slope at the bracket's middle xm; where that keeps f' away from
        // zero over the whole bracket (and its sign agrees with the ends'),
        // f has one root there, every halving of the bisection leads to it,
        // and the locate takes safeguarded FP32 Newton steps instead of
        // halvings, to the point where FP32 stops deciding the sign
        const float dm = 0.5f * (L + H);
        q = growth_f3_bounds(x0f + dm, rd3f, kf, &tf, physics);
        const float sl = 1.0f - dtpf * q.dg;
        const float reach = 0.5f * (H - L) + 1.2e-7f * x0f;
        mono = fabsf(sl) > 1.001f * dtpf * (q.edg + q.curv * reach) && (sl > 0.0f) != plo;
        float d = dm;
        for (int k = 0; mono && k < 48; ++k) {
            const float f = d - dtpf * q.g;
            if (!(fabsf(f) > 2.4e-7f * fabsf(d) + 4.0f * dtpf * q.err)) {
                mu = d;
                undecided = true;
                break;
            }
            if ((f > 0.0f) == plo) L = d;
            else H = d;
            float dn = d - f / (1.0f - dtpf * q.dg);
            if (!(dn > L && dn < H)) dn = 0.5f * (L + H);
            if (!(dn > L && dn < H)) break;  // the bracket is down to adjacent floats
            d = dn;
            // with the bounds: where the locate stops here, they are the
            // polish's slope bounds at mu and need no second evaluation
            q = growth_f3_bounds(x0f + d, rd3f, kf, &tf, physics);
        }
    }
    S.mono = mono;
    for (int k = 0; !mono && k < 64; ++k) {
        const float d = 0.5f * (L + H);
        if (!(d > L && d < H)) break;
        const GF q = growth_f3_call(x0f + d, rd3f, kf, &tf, physics);
        const float f = d - dtpf * q.g;
        if (!(fabsf(f) > 2.4e-7f * fabsf(d) + 4.0f * dtpf * q.err)) {
            mu = d;
            undecided = true;
            break;
        }
        if ((f > 0.0f) == plo) L = d;
        else H = d;
    }
    S.plo = plo;
    S.undecided = undecided;
    S.Lu = L;
    S.Hu = H;
    if (!undecided) mu = 0.5f * (L + H);
    S.mu = mu;
    // f' at mu for the first Newton step (D_eff's variation included)
    const float xs = x0f + mu;
    const GF qs = CERT && mono && undecided ? q : growth_f3_slope<CERT>(xs, rd3f, kf, &tf, physics);
    const float dg = qs.dg;
    if (CERT) {
        S.es = dtp * (double)qs.edg;
        S.cv = dtp * (double)qs.curv;
        S.xsp = (double)xs;
    }
    // 2. the polish starts at mu inside [lo, hi]
    double lo = x0 + (double)L, hi = x0 + (double)H;
    if (!(lo >= S.a)) lo = S.a;
    if (!(hi <= S.b)) hi = S.b;
    double xk = x0 + (double)mu;
    S.mu_inside = xk > lo && xk < hi;
    if (!S.mu_inside) xk = 0.5 * (lo + hi);
    S.lo = lo;
    S.hi = hi;
    S.xk = xk;
    S.xp = S.fp = 0.0;
    S.slope = 1.0 - dtp * (double)dg;  // Newton with the FP32 derivative first
    S.sdx = S.sdf = 1.0;
    S.have_slope = true;
    S.pmu = false;
    S.k = 0;
}

// A Newton step xn = xb - f(xb)/s with the FP32 slope s, f(xb) known to
// +-efb: between xb and the root f' differs from s by at most
// ds = es + cv (|xsp - xb| + 2 |xn - xb|), so (mean value theorem) the root
// lies within (|xn - xb| ds + efb) / (|s| - ds) of xn.  Certified when that
// is below 2^-43 xn (1.1e-13 of it, nearly nine times inside the 1e-12 bar).
//
// efb: an FP64 evaluation of f carries at most a few ulps of the terms whose
// difference it is (the sums of rho_v and rho_o, each a product of a handful
// of correctly rounded factors and exp, whose error CUDA bounds by 1 ulp);
// the callers allow 16 ulps (2^-49) of them.
// 1/s for the certified Newton steps without an FP64 division: the FP32
// reciprocal (within 2^-23 of 1/s) and one Newton iteration, within 2^-45;
// newton_certified counts that as a slope error of 2^-44 |s|.
SDM_HD double rcp_slope(double s) {
    const double r0 = (double)(1.0f / (float)s);
    return r0 * fma(-s, r0, 2.0);
}

SDM_HD bool newton_certified(const FastSolve &S, double xb, double xn, double efb) {
    const double step = fabs(xn - xb), as = fabs(S.slope);
    const double ds = S.es + S.cv * (fabs(S.xsp - xb) + 2.0 * step) + 0x1p-44 * as;
    if (!(ds < 0.25 * as)) return false;
    return step * ds + efb <= 0x1p-43 * xn * (as - ds);
}

// fs_replay is defined below; a certified step from x0 replays the halvings.
SDM_HD double fs_replay(FastSolve &S, double r, const Thermo &t, const ThermoF &tf, double dtp, int physics,
                        SolveCounters &cnt);

// After g0 = g(x0) in FP64: the paper's bracket and Euler test exactly, then
// the locate.  Returns true when the solve is finished (S.x1 set).  CERT: a
// certified Newton step from x0 finishes it too.
template <bool CERT>
SDM_HD bool fs_after_ends(FastSolve &S, double g0, bool pa, bool pb, GF q0, const Thermo &t, const ThermoF &tf,
                          double dtp, int physics, SolveCounters &cnt);

// DEFER (staged layout): where an end's sign needs the term-by-term FP64
// residual (fres_rare), the solve stops with that end in S.pend, the decided
// signs in S.pe0, S.pe1 and g0 in S.x1, and returns false; fs_resume_ends
// takes it from there in the next round, so that the few records that need
// it share warps instead of holding up the others.
template <bool CERT, bool DEFER = false>
SDM_HD bool fs_after_g0(FastSolve &S, double g0, const Thermo &t, const ThermoF &tf, double dtp, int physics,
                        SolveCounters &cnt) {
    const double x0 = S.x0;
    const double xa = x0 + fmin(2.0 * dtp * g0, 0.0);
    const float rd3f = (float)S.rd3, kf = (float)S.kappa, dtpf = (float)dtp, x0f = (float)x0;
    // a = max(r_d^2, xa); CERT: r_d^2 in FP64 only where the FP32 cube root
    // (1 ulp, squared: within 2^-20) cannot place it below xa
    double a;
    if (CERT) {
        float rd2f = cbrtf(rd3f);
        rd2f *= rd2f;
        a = xa > (double)rd2f * (1.0 + 0x1p-20) ? xa : fmax(rd2_of(S.rd3), xa);
    } else {
        a = fmax(rd2_of(S.rd3), xa);
    }
    const double b = x0 + fmax(2.0 * dtp * g0, 0.0);
    S.a = a;
    S.b = b;
    if (DEFER) S.pend = 0;
    // the ends' signs; at x0 itself f = -dtp g0 exactly.  The sign of f at
    // x0 + d (d an FP32 increment) is computed in FP32 and trusted where |f|
    // exceeds its error bound (it is then the sign an FP64 evaluation gives).
    // CERT: first from the FP32 slope at x0.  With D = xe - x0 (exact: xe is
    // within x0/16 of x0), f(xe) = D - dt' g0 - dt' g'(xi) D for some xi
    // between them, and g'(xi) lies within B = edg + curv (|D| + |x0 - x0f|)
    // of the FP32 slope dg; the sign is taken where the linear value clears
    // that, its own rounding and the rounding of an FP64 evaluation of f
    // (2^-46 of the terms' size mag).  Near equilibrium g0 is too small for
    // FP32 to sign f at either end, and this saves the FP64 evaluation there.
    GF q0;
    if (CERT) q0 = growth_f3_slope<CERT>(x0f, rd3f, kf, &tf, physics);
    bool pe[2];
    for (int e = 0; e < 2; ++e) {
        const double xe = e ? b : a;
        if (xe == x0) {
            pe[e] = -dtp * g0 > 0.0;
            continue;
        }
        if (CERT) {
            const double D = xe - x0;
            if (fabs(D) <= 0.0625 * x0) {
                const double lin = dtp * (double)q0.dg * D;
                const double F = (D - dtp * g0) - lin;
                const double B = (double)q0.edg + (double)q0.curv * (fabs(D) + fabs(x0 - (double)x0f));
                const double M = dtp * B * fabs(D) + 0x1p-48 * (fabs(D) + dtp * fabs(g0) + fabs(lin)) +
                                 0x1p-46 * dtp * (double)q0.mag;
                if (fabs(F) > M) {
                    pe[e] = F > 0.0;
                    continue;
                }
            }
        }
        {
            const float d = (float)(xe - x0);
            const GF q = growth_f3_call(x0f + d, rd3f, kf, &tf, physics);
            const float f = d - dtpf * q.g;
            if (fabsf(f) > 2.4e-7f * fabsf(d) + 4.0f * dtpf * q.err) {
                pe[e] = f > 0.0f;
            } else if (DEFER) {
                S.pend |= (uint8_t)(1 << e);
                pe[e] = false;
            } else {
                pe[e] = fres_rare(xe, x0, S.rd3, S.kappa, &t, dtp, physics) > 0.0;
            }
        }
    }
    if (DEFER && S.pend) {
        S.pe0 = pe[0];
        S.pe1 = pe[1];
        S.x1 = g0;
        return false;
    }
    return fs_after_ends<CERT>(S, g0, pe[0], pe[1], q0, t, tf, dtp, physics, cnt);
}

// The deferred ends' signs from the term-by-term FP64 residual, then the
// rest of fs_after_g0.
template <bool CERT>
SDM_HD bool fs_resume_ends(FastSolve &S, const Thermo &t, const ThermoF &tf, double dtp, int physics,
                           SolveCounters &cnt) {
    bool pe[2] = {S.pe0, S.pe1};
    for (int e = 0; e < 2; ++e)
        if (S.pend & (1 << e)) pe[e] = fres_rare(e ? S.b : S.a, S.x0, S.rd3, S.kappa, &t, dtp, physics) > 0.0;
    S.pend = 0;
    GF q0;
    if (CERT) q0 = growth_f3_slope<CERT>((float)S.x0, (float)S.rd3, (float)S.kappa, &tf, physics);
    return fs_after_ends<CERT>(S, S.x1, pe[0], pe[1], q0, t, tf, dtp, physics, cnt);
}

// After the signs pa, pb of f at the bracket's ends a = S.a, b = S.b: the
// Euler step, the bisection's first exit, or the setup of the polish (CERT:
// q0, the FP32 slope and its bounds at x0, is given).
template <bool CERT>
SDM_HD bool fs_after_ends(FastSolve &S, double g0, bool pa, bool pb, GF q0, const Thermo &t, const ThermoF &tf,
                          double dtp, int physics, SolveCounters &cnt) {
    const double x0 = S.x0, a = S.a, b = S.b;
    const float rd3f = (float)S.rd3, kf = (float)S.kappa, x0f = (float)x0;
    const bool pe[2] = {pa, pb};
    if (pe[0] == pe[1]) {  // f keeps its strict sign: the Euler step
        cnt.euler++;
        S.x1 = 0.5 * (a + b);
        return true;
    }
    if (b - a <= 0x1p-52 * b) {  // the bisection's own first exit
        S.x1 = 0.5 * (a + b);
        return true;
    }
    // x0 is an end of the bracket and f(x0) = -dt' g0 is known: the polish
    // starts at the Newton step from it (with the FP32 f').  These are the
    // solves whose g0 FP32 could not sign, close to equilibrium, where the
    // bracket is narrow and the step lands near the root; the replay starts
    // from the whole bracket.  x0 is not a secant point: g0 was formed as
    // growth() forms it, the polish residuals in the one-division form, and
    // over a step of a few ulps their difference is rounding.
    S.plo = pe[0];
    S.undecided = true;
    S.mono = false;
    S.Lu = (float)(a - x0);
    S.Hu = (float)(b - x0);
    S.mu = 0.0f;
    S.mu_inside = false;
    S.pmu = false;
    S.lo = a;
    S.hi = b;
    if (!CERT) q0 = growth_f3_slope<CERT>(x0f, rd3f, kf, &tf, physics);
    S.slope = 1.0 - dtp * (double)q0.dg;
    S.have_slope = true;
    S.sdx = S.sdf = 1.0;
    const double f0 = -dtp * g0;
    double xk = S.slope > 0.0 ? x0 - f0 * (CERT ? rcp_slope(S.slope) : 1.0 / S.slope) : 0.5 * (a + b);
    const bool newton = xk > a && xk < b;
    if (!newton) xk = 0.5 * (a + b);
    S.xp = S.fp = 0.0;
    S.xk = xk;
    S.k = 0;
    if (CERT) {
        // the Newton step from x0 is the result where its certified error is
        // far below 1e-12: f(x0) = -dt' g0 is known to the rounding of g0's
        // terms (their size mag, from FP32); the replay then checks that the
        // bisection's halvings lead to it
        S.es = dtp * (double)q0.edg;
        S.cv = dtp * (double)q0.curv;
        S.xsp = x0;
        // f strictly monotone on [a, b] (its slope bounds as in fs_locate):
        // one root, to which every halving leads, and no replay
        const double reach = fmax(x0 - a, b - x0) + fabs(x0 - (double)x0f);
        S.mono = b - a <= 0.0625 * x0 && fabs(S.slope) > 1.001 * (S.es + S.cv * reach) &&
                 (S.slope > 0.0) != S.plo;
        if (newton && newton_certified(S, x0, xk, 0x1p-49 * dtp * (double)q0.mag)) {
            cnt.certified++;
            S.x1 = S.mono ? xk : fs_replay(S, xk, t, tf, dtp, physics, cnt);
            return true;
        }
    }
    return false;
}

// How a solve starts, decided from g(x0) in FP32:
enum { kStartPolish = 0, kStartEuler = 1, kStartTiny = 2, kStartExact = 3 };
// kStartPolish: f changes sign over the bracket; the locate is done and the
//   first FP64 evaluation is the polish's.
// kStartEuler, kStartTiny: the Euler step, or a bracket below FP64
//   resolution; x1 = (a + b)/2 needs g(x0) in FP64.
// kStartExact: FP32 cannot decide; the paper's path from g(x0) in FP64.
//
// With g0 known to +-e0, the moving end of the bracket x0 + 2 dt' g0 is
// known to +-u; the sign of f there is trusted only where |f| exceeds the
// FP32 bound plus |f'| u, so every decision taken here is the one the FP64
// bracket gives.  Only the Euler step, whose result is g(x0) itself, then
// needs g(x0) in FP64: the other solves save that evaluation.
template <bool CERT>
SDM_HD int fs_start(FastSolve &S, const ThermoF &tf, double dtp, int physics) {
    const double x0 = S.x0;
    const float rd3f = (float)S.rd3, kf = (float)S.kappa, dtpf = (float)dtp, x0f = (float)x0;
    const GF q0 = growth_f3_call(x0f, rd3f, kf, &tf, physics);
    if (!(fabsf(q0.g) > q0.err)) return kStartExact;  // the sign of g0
    const bool grow = q0.g > 0.0f;
    const float dE = 2.0f * dtpf * q0.g;                          // the moving end's increment
    const float u = 2.0f * dtpf * q0.err + 2.4e-7f * fabsf(dE);   // and its uncertainty
    float rd2f = cbrtf(rd3f);
    rd2f *= rd2f;
    const float rtol = 1e-6f * rd2f;
    // the sign of f at x0 + d, d known to +-ud; ok = decided
    auto sign_at = [&](float d, float ud, bool *ok) -> bool {
        const GF q = growth_f3<kDgKoehler>(x0f + d, rd3f, kf, tf, physics);
        const float f = d - dtpf * q.g;
        const float fpr = 1.0f + 2.0f * dtpf * (fabsf(q.dg) + fabsf(q.g) / (x0f + d));  // >= |f'|
        *ok = fabsf(f) > 2.4e-7f * fabsf(d) + 4.0f * dtpf * q.err + fpr * ud;
        return f > 0.0f;
    };
    bool ok, pa, pb;
    float L, H;
    S.clamp = false;
    if (grow) {  // a = max(r_d^2, x0) = x0 with f(x0) = -dt' g0 < 0; b = x0 + dE
        if (!(x0f > rd2f + rtol)) return kStartExact;
        pa = false;
        pb = sign_at(dE, u, &ok);
        if (!ok) return kStartExact;
        L = 0.0f;
        H = dE;
        S.a = x0;
        S.b = x0 + (double)dE;
    } else {  // b = x0 with f(x0) > 0; a = max(r_d^2, x0 + dE)
        pb = true;
        const double xa = x0 + (double)dE;
        if (xa > (double)(rd2f + rtol) + (double)u) {
            pa = sign_at(dE, u, &ok);
            L = dE;
            S.a = xa;
        } else if (xa < (double)(rd2f - rtol) - (double)u) {
            S.clamp = true;
            S.rd2 = rd2_of(S.rd3);
            L = (float)(S.rd2 - x0);
            pa = sign_at(L, 0.0f, &ok);
            S.a = S.rd2;
        } else {
            return kStartExact;
        }
        if (!ok) return kStartExact;
        H = 0.0f;
        S.b = x0;
    }
    if (pa == pb) return kStartEuler;
    // the bisection's own first exit, b - a <= 2^-52 b
    const double w = (double)(H - L), uw = S.clamp ? 0.0 : (double)u;
    if (w + uw <= 0x1p-52 * (S.b - uw)) return kStartTiny;
    if (!(w - uw > 0x1p-52 * (S.b + uw))) return kStartExact;
    fs_locate<CERT>(S, L, H, pa, tf, dtp, physics);
    return kStartPolish;
}

// x1 of the Euler step (or of a bracket below resolution) from g0 in FP64:
// the paper's (a + b)/2, with the clamp of a that fs_start decided
SDM_HD double fs_euler(const FastSolve &S, double g0, double dtp) {
    const double x0 = S.x0;
    const double a = S.clamp ? S.rd2 : x0 + fmin(2.0 * dtp * g0, 0.0);
    const double b = x0 + fmax(2.0 * dtp * g0, 0.0);
    return 0.5 * (a + b);
}

// 3. replay: near activation f need not be monotonic, and a bracket can hold
//    several roots.  The polish found the one nearest mu; the bisection takes
//    the one its halvings lead to.  Replaying those halvings from the bracket
//    where FP32 stopped deciding (in FP32, and in FP64 wherever FP32 cannot
//    tell away from r) checks that they lead to r; where they leave it, the
//    exact bisection takes over.  Returns the solve's result.
SDM_HD double fs_replay(FastSolve &S, double r, const Thermo &t, const ThermoF &tf, double dtp, int physics,
                        SolveCounters &cnt) {
    const double x0 = S.x0;
    const float rd3f = (float)S.rd3, kf = (float)S.kappa, dtpf = (float)dtp, x0f = (float)x0;
    // dr carries r - x0 to FP32: points within a few of its ulps, or within a
    // few FP64 ulps of r itself (the signs are taken at FP64 points), are
    // taken as r
    const float dr = (float)(r - x0);
    const float dtol = fmaxf(4.0f * 5.9604645e-8f * fabsf(dr), (float)(0x1p-50 * r));
    const bool plo = S.plo;
    float RL = S.Lu, RH = S.Hu;
    if (S.mu_inside) {
        if (!(fabsf(S.mu - dr) <= dtol || (S.pmu == plo) == (S.mu < dr))) {
            cnt.fallback++;
            return bisect_rest(S.pmu == plo ? fmax(S.a, x0 + (double)S.mu) : fmax(S.a, x0 + (double)RL),
                               S.pmu == plo ? fmin(S.b, x0 + (double)RH) : fmin(S.b, x0 + (double)S.mu), plo,
                               x0, S.rd3, S.kappa, t, dtp, physics);
        }
        if (S.pmu == plo) RL = S.mu;
        else RH = S.mu;
    }
    for (int it = 0; it < 64; ++it) {
        const float m = 0.5f * (RL + RH);
        if (!(m > RL && m < RH) || fabsf(m - dr) <= dtol) break;
        const GF q = growth_f3_call(x0f + m, rd3f, kf, &tf, physics);
        const float f = m - dtpf * q.g, nz = 2.4e-7f * fabsf(m) + 4.0f * dtpf * q.err;
        bool pm = f > 0.0f;
        if (!(fabsf(f) > nz)) {
            // within a few noise widths of r: the halvings close in on r
            const double sl = fabs(S.have_slope ? S.slope : S.sdf / S.sdx);
            if ((double)fabsf(m - dr) * sl <= 8.0 * (double)nz) break;
            pm = fres_rare(x0 + (double)m, x0, S.rd3, S.kappa, &t, dtp, physics) > 0.0;
        }
        if (pm == plo) RL = m;
        else RH = m;
        if (pm != (plo == (m < dr))) {
            cnt.fallback++;
            return bisect_rest(fmax(S.a, x0 + (double)RL), fmin(S.b, x0 + (double)RH), plo, x0, S.rd3, S.kappa,
                               t, dtp, physics);
        }
    }
    return r;
}

// After v = growth_eval(S.xk, false, .., &mag): one polish step (bracketed
// Newton, then secant, in FP64 with exact signs).  Returns true when the solve is
// finished (S.x1 set).  CERT: the first Newton step also settles where it is
// certified (newton_certified).
template <bool CERT>
SDM_HD bool fs_after_polish(FastSolve &S, double v, double mag, const Thermo &t, const ThermoF &tf, double dtp,
                            int physics, SolveCounters &cnt) {
    const double xk = S.xk, fk = xk - S.x0 - dtp * v;
    // f(xk) within the rounding of its own evaluation (16 ulps of its terms)
    const bool at_noise = fabs(fk) <= 0x1p-48 * (fabs(xk - S.x0) + dtp * mag);
    const int k = S.k;
    if (k == 0) S.pmu = fk > 0.0;
    double r = 0.0;
    bool settled = false;
    if (fk == 0.0) {
        r = xk;
        settled = true;
    } else {
        if ((fk > 0.0) == S.plo) S.lo = xk;
        else S.hi = xk;
        if (S.hi - S.lo <= 0x1p-46 * S.hi) {
            r = 0.5 * (S.lo + S.hi);
            settled = true;
        }
    }
    if (!settled && k < 12) {
        const double lo = S.lo, hi = S.hi;
        const bool secant = k > 0 && fk != S.fp;
        double xn;
        if (secant) {
            S.sdx = xk - S.xp;
            S.sdf = fk - S.fp;
            xn = xk - fk * (S.sdx / S.sdf);
            S.have_slope = false;
        } else {
            xn = S.slope != 0.0 ? xk - fk * (CERT ? rcp_slope(S.slope) : 1.0 / S.slope) : 0.5 * (lo + hi);
        }
        // the secant converges superlinearly: once its step is below 2^-30 x
        // the error left is of order (2^-30)(previous step) x, far below
        // 2^-46 x; a Newton step with the approximate FP32 derivative must
        // itself be that small.  A step onto the end of the bracket that xk
        // has just become (a correction below one ulp) settles only when
        // f(xk) is at the rounding level of its evaluation: near it a secant
        // slope from close points is itself rounding.
        const bool inside = at_noise ? xn >= lo && xn <= hi : xn > lo && xn < hi;
        // certified: f(xk) carries the rounding of the one-division form (of
        // its terms xk - x0 and dt' g's, mag)
        const bool small = fabs(xn - xk) <= (secant ? 0x1p-30 : 0x1p-46) * xk;
        const bool cert = CERT && !small && !secant && S.have_slope &&
                          newton_certified(S, xk, xn, 0x1p-49 * (fabs(xk - S.x0) + dtp * mag));
        if (inside && (small || cert)) {
            if (cert) cnt.certified++;
            r = xn;
            settled = true;
        } else {
            // a larger step past an end of the bracket says the root hugs that
            // end: move 1/64 in from it
            if (!(xn < hi)) xn = hi - (hi - lo) * 0.015625;
            if (!(xn > lo)) xn = lo + (hi - lo) * 0.015625;
            S.xp = xk;
            S.fp = fk;
            S.xk = xn;
            S.k = k + 1;
            return false;
        }
    }
    if (!settled) {  // did not settle in 13 evaluations
        cnt.fallback++;
        S.x1 = bisect_rest(S.lo, S.hi, S.plo, S.x0, S.rd3, S.kappa, t, dtp, physics);
        return true;
    }
    S.x1 = S.undecided && !(CERT && S.mono) ? fs_replay(S, r, t, tf, dtp, physics, cnt) : r;
    return true;
}

// the whole fast solve for one super-droplet
template <bool CERT = false>
__host__ __device__ double solve_rw2_fast(double x0, double rd3, double kappa, const Thermo &t,
                                          const ThermoF &tf, double dtp, int physics, SolveCounters &cnt) {
    FastSolve S;
    S.x0 = x0;
    S.rd3 = rd3;
    S.kappa = kappa;
    // The first FP64 evaluation is g(x0) where the start needs it (an Euler
    // step, or FP32 could not decide), else the polish's first; then one per
    // polish step, all through one call site.
    const int start = fs_start<CERT>(S, tf, dtp, physics);
    for (int k = 0; k < 15; ++k) {
        const bool g0 = k == 0 && start != kStartPolish;
        cnt.evals++;
        double mag;
        const double v = growth_eval<CERT>(g0 ? x0 : S.xk, g0, rd3, kappa, t, physics, &mag, &tf);
        if (g0) {
            if (start == kStartExact) {
                if (fs_after_g0<CERT>(S, v, t, tf, dtp, physics, cnt)) return S.x1;
                continue;
            }
            if (start == kStartEuler) cnt.euler++;
            return fs_euler(S, v, dtp);
        }
        if (fs_after_polish<CERT>(S, v, mag, t, tf, dtp, physics, cnt)) return S.x1;
    }
    return S.x1;  // not reached: the polish finishes within 13 evaluations
}

// ---------------------------------------------------------------------------
// Mixed-precision solve: the same bracket and Euler rule, then a bracketed
// Newton iteration, all in FP32 on the increment d = x - x0 (so that a small
// change of a large r_w^2 is not lost to FP32 rounding of x itself).  The
// new r_w^2 = x0 + d is formed in FP64.  Iterates never leave the bracket;
// after 24 steps without settling the last one is used.
__host__ __device__ bool solve_rw2_f32(double x0, double rd3, double kappa, const ThermoF &tf,
                                       float dtp, int physics, double *x1, SolveCounters &cnt) {
    const float rd3f = (float)rd3, kf = (float)kappa;
    const float g0 = growth_f3_call((float)x0, rd3f, kf, &tf, physics).g;
    const float rdf = cbrtf(rd3f);
    const float lo_d = fmaxf((float)((double)(rdf * rdf) - x0), fminf(2.0f * dtp * g0, 0.0f));
    const float hi_d = fmaxf(2.0f * dtp * g0, 0.0f);
    auto f = [&](float d, float *der) -> float {
        const GF q = growth_f3<kDgKoehler>((float)(x0 + (double)d), rd3f, kf, tf, physics);
        if (der) *der = 1.0f - dtp * q.dg;
        return d - dtp * q.g;
    };
    const float fa = f(lo_d, nullptr), fb = f(hi_d, nullptr);
    if ((fa > 0.0f) == (fb > 0.0f)) {
        cnt.euler++;
        *x1 = x0 + 0.5 * ((double)lo_d + (double)hi_d);
        return true;
    }
    float lo = lo_d, hi = hi_d;
    const bool plo = fa > 0.0f;
    float d = 0.5f * (lo + hi);
    for (int k = 0; k < 24; ++k) {
        float der;
        const float fd = f(d, &der);
        if (fd == 0.0f) break;
        if ((fd > 0.0f) == plo) lo = d;
        else hi = d;
        float dn = der != 0.0f ? d - fd / der : 0.5f * (lo + hi);
        if (!(dn > lo && dn < hi)) dn = 0.5f * (lo + hi);
        const float step = fabsf(dn - d);
        d = dn;
        // settled to FP32 resolution of r_w^2 itself (not of the increment)
        const float tol = 2.4e-7f * (float)x0;
        if (step <= tol || hi - lo <= tol) {
            *x1 = x0 + (double)d;
            return true;
        }
    }
    *x1 = x0 + (double)d;
    return true;
}

// FP32 is kept away from droplets near Koehler activation in supersaturated
// air, where the growth equation is stiff and the root sensitive: there the
// FP64 solve runs.  r_crit^2 = 3 kappa r_d^3 / A (the kappa-Koehler critical
// radius for a dilute solution).
__host__ __device__ __forceinline__ bool near_activation(double x0, double rd3, double kappa,
                                                         const Thermo &t) {
    if (t.rho_v_eff < 0.99 * t.rho_vs) return false;
    const double rc2 = 3.0 * kappa * rd3 / t.A;
    return x0 < 9.0 * rc2;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// LPC lanes per cell (4, 8 or 32): each lane solves every LPC-th
// super-droplet of its cell, the group's lanes share the cell's
// thermodynamics and sum through shuffles inside the group.
// MODE: the solver, fixed at compile time so that each kernel carries only
// its own code.
enum { kModeBisect = 0, kModeFast = 1, kModeMixed = 2 };

template <int MODE>
__device__ __forceinline__ double solve_mode(double x0, double rd3, double kappa, const Thermo &t,
                                             const ThermoF &tf, double dtp, int physics, SolveCounters &cnt) {
    double x1;
    if (MODE == kModeMixed && !near_activation(x0, rd3, kappa, t)) {
        solve_rw2_f32(x0, rd3, kappa, tf, (float)dtp, physics, &x1, cnt);
    } else if (MODE == kModeBisect) {
        int eu = 0;
        x1 = solve_rw2_bisect(x0, rd3, kappa, t, dtp, physics, &eu);
        cnt.euler += eu;
    } else {
        x1 = solve_rw2_fast(x0, rd3, kappa, t, tf, dtp, physics, cnt);
    }
    return x1;
}

constexpr int kMaxBlock = 128;

// the per-substep thermodynamics out of line, like the solver's other
// once-per-cell or rare code, so that the FP64 growth loop stays compact
__device__ __noinline__ Thermo thermo_cond(double th, double rv, double rd, double RH_max, double rdf) {
    return thermo_eval_f<true>(th, rv, rd, RH_max, rdf);
}

// The ambient state the solve sees, per cell, into out: the same out-of-line
// thermodynamics the condensation kernel calls (what: 0 T, 1 p, 2 rho_vs,
// 3 RH = rho_v / rho_vs), p = rho_d (R_d + r_v R_v) T (Appendix A).
__global__ void k_cond_ambient(const double *th, const double *rv, const double *rhod, int n_cells, int what,
                               double *out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const Thermo t = thermo_cond(th[c], rv[c], rhod[c], 44.0, rhod_factor(rhod[c]));
    double v = t.T;
    if (what == 1) v = rhod[c] * (phys::R_d + rv[c] * phys::R_v) * t.T;
    else if (what == 2) v = t.rho_vs;
    else if (what == 3) v = t.rho_v / t.rho_vs;
    out[c] = v;
}

cudaError_t launch_cond_ambient(sdm_ctx *c, int what) {
    const int B = 128;
    k_cond_ambient<<<grid_for(c->grid.n_cells, B), B, 0, c->stream>>>(c->th, c->rv, c->rhod, c->grid.n_cells, what,
                                                                       c->outbuf);
    return cudaGetLastError();
}

// ORD: the warps take their work in order of decreasing cost (order),
// which the previous launch recorded per warp into cost (its FP64 growth
// evaluations, the bulk of a warp's time); see launch_condense_lpc.
// Results do not depend on the order: cells are independent.
template <int LPC, int MODE, bool ORD>
__global__ void __launch_bounds__(kMaxBlock) k_condense(SdArrays s, const uint32_t *offset, double *th, double *rv,
                           const double *rhod, Grid g, int sstp, double RH_max, int physics, DevStats *st,
                           const uint32_t *order, float *cost, int64_t n_warps) {
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (ORD && wid >= n_warps) return;  // whole warps only: the kernel syncs within warps
    const int64_t wmap = ORD ? (int64_t)order[wid] : wid;
    const int lane = threadIdx.x & 31;
    const int64_t gt = wmap * 32 + lane;
    const int sl = lane % LPC;
    const int64_t c64 = gt / LPC;
    const bool live = c64 < g.n_cells;
    const int c = live ? (int)c64 : 0;
    const uint32_t beg = live ? offset[c] : 0, end = live ? offset[c + 1] : 0;
    double thc = live ? th[c] : 289.0, rvc = live ? rv[c] : 0.0;
    const double rd = live ? rhod[c] : 1.0;
    const double dtp = g.dt / sstp;
    SolveCounters cnt{0, 0, 0, 0};
    bool bad = false;
    // the cell's ambient state for the solves sits in shared memory: read
    // there by reference it takes no registers across the solve
    __shared__ Thermo s_t[kMaxBlock / LPC];
    __shared__ ThermoF s_tf[kMaxBlock / LPC];
    constexpr int kQueueCap = 128;  // FP64 queue of the mixed one-cell-per-warp solve
    __shared__ uint32_t s_q[(MODE == kModeMixed && LPC == 32) ? kMaxBlock / 32 : 1][kQueueCap];
    const int gi = threadIdx.x / LPC;
    const Thermo &t = s_t[gi];
    const ThermoF &tf = s_tf[gi];
    const double rdf = rhod_factor(rd);
    for (int sub = 0; sub < sstp; ++sub) {
        {
            const Thermo tt = thermo_cond(thc, rvc, rd, RH_max, rdf);
            if (sl == 0) {
                s_t[gi] = tt;
                s_tf[gi] = to_float(tt);
            }
        }
        __syncwarp();
        double sum = 0.0;
        if constexpr (MODE == kModeMixed && LPC == 32) {
            // Mixed precision, one cell per warp: the FP32 solves first, in
            // rounds of 32 super-droplets; those near activation are queued
            // (in id order, by ballot) and then take the FP64 solve 32 at a
            // time, so that its lanes are full instead of scattered
            uint32_t *q = s_q[threadIdx.x >> 5];
            int nq = 0;
            for (uint32_t i0 = beg; i0 < end; i0 += 32) {
                const uint32_t i = i0 + lane;
                bool need64 = false;
                unsigned long long N = 0;
                if (i < end) N = s.N[i];
                if (N != 0) {
                    const double x0 = s.rw2[i], rd3 = s.rd3[i], kap = s.kappa[i];
                    need64 = near_activation(x0, rd3, kap, t);
                    if (!need64) {
                        double x1;
                        solve_rw2_f32(x0, rd3, kap, tf, (float)dtp, physics, &x1, cnt);
                        bad |= !isfinite(x1);
                        s.rw2[i] = x1;
                        sum += (double)N * (x1 * sqrt(x1) - x0 * sqrt(x0));
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, need64);
                if (need64) {
                    const int pos = nq + __popc(m & ((1u << lane) - 1u));
                    if (pos < kQueueCap) {
                        q[pos] = i;
                    } else {  // a cell far above its share: solve in place
                        const double x0 = s.rw2[i];
                        const double x1 = solve_rw2_fast(x0, s.rd3[i], s.kappa[i], t, tf, dtp, physics, cnt);
                        bad |= !isfinite(x1);
                        s.rw2[i] = x1;
                        sum += (double)N * (x1 * sqrt(x1) - x0 * sqrt(x0));
                    }
                }
                nq += __popc(m);
            }
            __syncwarp();
            const int nqs = nq < kQueueCap ? nq : kQueueCap;
            for (int k = lane; k < nqs; k += 32) {
                const uint32_t i = q[k];
                const unsigned long long N = s.N[i];
                const double x0 = s.rw2[i];
                const double x1 = solve_rw2_fast(x0, s.rd3[i], s.kappa[i], t, tf, dtp, physics, cnt);
                bad |= !isfinite(x1);
                s.rw2[i] = x1;
                sum += (double)N * (x1 * sqrt(x1) - x0 * sqrt(x0));
            }
        } else {
            for (uint32_t i = beg + sl; i < end; i += LPC) {
                const unsigned long long N = s.N[i];
                if (N == 0) continue;
                const double x0 = s.rw2[i];
                const double x1 = solve_mode<MODE>(x0, s.rd3[i], s.kappa[i], t, tf, dtp, physics, cnt);
                bad |= !isfinite(x1);
                s.rw2[i] = x1;
                sum += (double)N * (x1 * sqrt(x1) - x0 * sqrt(x0));
            }
        }
#pragma unroll
        for (int o = LPC / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        const double drv = -4.0 * phys::pi * phys::rho_w / (3.0 * g.dV * rd) * sum;
        rvc = t.rv + drv;
        thc = t.th + drv * t.dth_drv;
        __syncwarp();  // every lane has read s_t before the next substep writes it
    }
    bad |= live && (!isfinite(rvc) || !isfinite(thc));
    const unsigned ne = __reduce_add_sync(0xffffffffu, (unsigned)cnt.euler);
    const unsigned nf = __reduce_add_sync(0xffffffffu, (unsigned)cnt.fallback);
    const unsigned anybad = __any_sync(0xffffffffu, bad);
    const unsigned nev = ORD ? __reduce_add_sync(0xffffffffu, (unsigned)cnt.evals) : 0u;
    if (live && sl == 0) {
        th[c] = thc;
        rv[c] = rvc;
    }
    if (lane == 0) {
        if (ne) atomicAdd(&st->n_euler, (unsigned long long)ne);
        if (nf) atomicAdd(&st->n_fallback, (unsigned long long)nf);
        if (anybad) atomicOr(&st->flags, kFlagNumeric);
        if (ORD) cost[wmap] = (float)nev;
    }
}

// Longest work first: the warps' indices in order of decreasing cost, one
// block.  A counting sort on 256 cost buckets spread linearly between the
// smallest and the largest cost: the order within a bucket is whatever the
// atomics give, which is harmless, since the order never changes a result.
constexpr int kOrderMaxWarps = 8192, kOrderBuckets = 256;

__global__ void __launch_bounds__(1024) k_cond_order(const float *cost, uint32_t *order, int n) {
    __shared__ unsigned s_cnt[kOrderBuckets];
    __shared__ float s_lo[32], s_hi[32];
    float lo = INFINITY, hi = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float cv = fmaxf(cost[i], 0.0f);
        lo = fminf(lo, cv);
        hi = fmaxf(hi, cv);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        s_lo[threadIdx.x >> 5] = lo;
        s_hi[threadIdx.x >> 5] = hi;
    }
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    lo = s_lo[0];
    hi = s_hi[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        lo = fminf(lo, s_lo[w]);
        hi = fmaxf(hi, s_hi[w]);
    }
    const float scale = hi > lo ? (kOrderBuckets - 1) / (hi - lo) : 0.0f;
    // bucket 0 holds the most expensive warps
    auto bucket = [&](int i) {
        const int b = (int)((hi - fmaxf(cost[i], 0.0f)) * scale);
        return b < 0 ? 0 : (b >= kOrderBuckets ? kOrderBuckets - 1 : b);
    };
    for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&s_cnt[bucket(i)], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {  // exclusive scan of 256 counts
        unsigned run = 0;
        for (int b = 0; b < kOrderBuckets; ++b) {
            const unsigned c = s_cnt[b];
            s_cnt[b] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) order[atomicAdd(&s_cnt[bucket(i)], 1u)] = (uint32_t)i;
}

// Ensemble condensation, one substep: a block per tile (tiles never straddle
// two members), the member's thermodynamics computed once per block, a
// deterministic block sum of N (r_w^3[new] - r_w^3[old]) into tile_sum.
template <int MODE>
__global__ void k_ens_cond_tiles(SdArrays s, const MemberDev *M, const uint32_t *tile_member,
                                 const uint32_t *tile_beg, const uint32_t *tile_end, double *tile_sum,
                                 EnsCondParams p, DevStats *st) {
    __shared__ Thermo s_t;
    __shared__ double s_part[32];
    const int tile = blockIdx.x;
    const MemberDev &md = M[tile_member[tile]];
    __shared__ ThermoF s_tf;
    if (threadIdx.x == 0) {  // the single-context kernel's thermodynamics, the same code
        s_t = thermo_cond(md.th, md.rv, md.rhod, p.RH_max, rhod_factor(md.rhod));
        s_tf = to_float(s_t);
    }
    __syncthreads();
    const Thermo &t = s_t;
    const ThermoF &tf = s_tf;
    const double dtp = p.dt / p.sstp;
    SolveCounters cnt{0, 0, 0, 0};
    double sum = 0.0;
    bool bad = false;
    for (uint32_t i = tile_beg[tile] + threadIdx.x; i < tile_end[tile]; i += blockDim.x) {
        const unsigned long long N = s.N[i];
        if (N == 0) continue;
        const double x0 = s.rw2[i];
        const double x1 = solve_mode<MODE>(x0, s.rd3[i], s.kappa[i], t, tf, dtp, p.physics, cnt);
        bad |= !isfinite(x1);
        s.rw2[i] = x1;
        sum += (double)N * (x1 * sqrt(x1) - x0 * sqrt(x0));
    }
    sum = warp_sum(sum);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) s_part[w] = sum;
    const unsigned ne = __reduce_add_sync(0xffffffffu, (unsigned)cnt.euler);
    const unsigned nf = __reduce_add_sync(0xffffffffu, (unsigned)cnt.fallback);
    const unsigned anybad = __any_sync(0xffffffffu, bad);
    __syncthreads();
    if (threadIdx.x == 0) {
        double tsum = 0.0;
        for (int v = 0; v < (int)(blockDim.x >> 5); ++v) tsum += s_part[v];
        tile_sum[tile] = tsum;
    }
    if (lane == 0) {
        if (ne) atomicAdd(&st->n_euler, (unsigned long long)ne);
        if (nf) atomicAdd(&st->n_fallback, (unsigned long long)nf);
        if (anybad) atomicOr(&st->flags, kFlagNumeric);
    }
}

// the largest block the ensemble condensation kernel of this mode launches
// with (its register count bounds it)
int ens_cond_max_threads(const EnsCondParams &p) {
    cudaFuncAttributes a{};
    cudaError_t e;
    if (p.mixed) e = cudaFuncGetAttributes(&a, k_ens_cond_tiles<kModeMixed>);
    else if (p.solver == 0) e = cudaFuncGetAttributes(&a, k_ens_cond_tiles<kModeBisect>);
    else e = cudaFuncGetAttributes(&a, k_ens_cond_tiles<kModeFast>);
    return e == cudaSuccess ? a.maxThreadsPerBlock : 128;
}

cudaError_t launch_ens_cond_tiles(SdArrays s, const MemberDev *M, const uint32_t *tile_member,
                                  const uint32_t *tile_beg, const uint32_t *tile_end, double *tile_sum,
                                  int n_tiles, int threads, EnsCondParams p, DevStats *st,
                                  cudaStream_t stream) {
    if (n_tiles == 0) return cudaSuccess;
    if (p.mixed)
        k_ens_cond_tiles<kModeMixed><<<n_tiles, threads, 0, stream>>>(s, M, tile_member, tile_beg, tile_end,
                                                                      tile_sum, p, st);
    else if (p.solver == 0)
        k_ens_cond_tiles<kModeBisect><<<n_tiles, threads, 0, stream>>>(s, M, tile_member, tile_beg, tile_end,
                                                                       tile_sum, p, st);
    else
        k_ens_cond_tiles<kModeFast><<<n_tiles, threads, 0, stream>>>(s, M, tile_member, tile_beg, tile_end,
                                                                     tile_sum, p, st);
    return cudaGetLastError();
}

// Where the launch is only a few waves of warps, the last wave decides the
// time: one warp's solves take a sizeable part of the whole (2D case: about
// 3 ms of 8).  There the warps run longest-first, in the order of their cost
// in the previous launch (the cells change slowly from step to step); with
// many waves (or no cost yet) the order is the cells' own.
template <int LPC, int MODE>
static int launch_condense_lpc(sdm_ctx *c, const sdm_opts &o, int B) {
    const int64_t threads = ((int64_t)c->grid.n_cells * LPC + 31) / 32 * 32;
    const int64_t n_warps = threads / 32;
    if (LPC == 32 && c->cond_order_on && n_warps <= kOrderMaxWarps) {
        if (c->cond_nw != n_warps) {
            cudaFree(c->cond_order);
            cudaFree(c->cond_cost);
            c->cond_order = nullptr;
            c->cond_cost = nullptr;
            c->cond_nw = 0;
            if (cudaMalloc(&c->cond_order, 4 * n_warps) == cudaSuccess &&
                cudaMalloc(&c->cond_cost, 4 * n_warps) == cudaSuccess &&
                cudaMemsetAsync(c->cond_cost, 0, 4 * n_warps, c->stream) == cudaSuccess)
                c->cond_nw = n_warps;
            cudaGetLastError();
        }
        if (c->cond_nw == n_warps) {
            k_cond_order<<<1, 1024, 0, c->stream>>>(c->cond_cost, c->cond_order, (int)n_warps);
            k_condense<LPC, MODE, LPC == 32><<<grid_for(threads, B), B, 0, c->stream>>>(
                c->buf[c->cur], c->offset, c->th, c->rv, c->rhod, c->grid, o.sstp_cond, o.RH_max, c->oi.physics,
                c->dstats, c->cond_order, c->cond_cost, n_warps);
            return 2;
        }
    }
    k_condense<LPC, MODE, false><<<grid_for(threads, B), B, 0, c->stream>>>(
        c->buf[c->cur], c->offset, c->th, c->rv, c->rhod, c->grid, o.sstp_cond, o.RH_max, c->oi.physics,
        c->dstats, nullptr, nullptr, n_warps);
    return 1;
}

template <int MODE>
static int launch_condense_mode(sdm_ctx *c, const sdm_opts &o, int lpc, int B) {
    if (lpc == 4) return launch_condense_lpc<4, MODE>(c, o, B);
    if (lpc == 8) return launch_condense_lpc<8, MODE>(c, o, B);
    return launch_condense_lpc<32, MODE>(c, o, B);
}

// ---------------------------------------------------------------------------
// Staged condensation (FP64, fast solver), for domains of many cells: each
// substep is a chain of small kernels instead of one kernel that carries a
// super-droplet's whole solve.  (1) the cells' ambient state; (2) every
// super-droplet's FP32 start (fs_start), its solve state written to a record;
// (3) rounds of FP64 growth evaluations over compacted lists of the records
// that still need one, each round one evaluation per record (so the lanes of
// a warp do the same work), finished solves writing their r_w^2; (4) per
// cell, the sum of eq. rhov_update and the update of r_v and theta.  The
// solve's steps are those of solve_rw2_fast<true>: the fused kernel's fast
// solve, which also settles on a certified Newton step, signs the bracket's
// ends from the FP32 slope near equilibrium and takes tiny ventilation
// corrections in FP32 (each within 1e-12 of the bisection's root, like the
// fused solve).  The solve state travels through HBM between the kernels,
// which the FP64-bound fused kernel leaves idle.
enum { kTaskNone = 0, kTaskG0Euler = 1, kTaskG0Tiny = 2, kTaskG0Exact = 3, kTaskPolish = 4, kTaskG0End = 5 };
// kTaskG0End: g(x0) done, a bracket end's sign deferred (fs_resume_ends)

struct StagedRec {
    FastSolve S;
    uint32_t sd;
    int task;
};

// the first task of a solve from its start class
SDM_HD int cs_task_of(int st) {
    return st == kStartPolish  ? kTaskPolish
           : st == kStartExact ? kTaskG0Exact
           : st == kStartEuler ? kTaskG0Euler
                               : kTaskG0Tiny;
}

// One round of a staged solve: one FP64 growth evaluation (or, for a
// deferred bracket end, its term-by-term residual) and the step it feeds.
// Returns true when the solve is finished (S.x1 set); task becomes the next
// round's.  The host build runs the same sequence (tests/hostcheck).
SDM_HD bool cs_step(int &task, FastSolve &S, const Thermo &t, const ThermoF &tf, double dtp, int physics,
                    SolveCounters &cnt) {
    cnt.evals++;
    if (task == kTaskG0End) {  // the deferred ends' FP64 residuals
        const bool done = fs_resume_ends<true>(S, t, tf, dtp, physics, cnt);
        if (!done) task = kTaskPolish;
        return done;
    }
    const bool g0 = task != kTaskPolish;
    double mag;
    const double v = growth_eval<true>(g0 ? S.x0 : S.xk, g0, S.rd3, S.kappa, t, physics, &mag, &tf);
    if (task == kTaskG0Euler || task == kTaskG0Tiny) {
        if (task == kTaskG0Euler) cnt.euler++;
        S.x1 = fs_euler(S, v, dtp);
        return true;
    }
    if (task == kTaskG0Exact) {
        const bool done = fs_after_g0<true, true>(S, v, t, tf, dtp, physics, cnt);
        if (!done) task = S.pend ? kTaskG0End : kTaskPolish;
        return done;
    }
    return fs_after_polish<true>(S, v, mag, t, tf, dtp, physics, cnt);
}

struct StagedCell {
    Thermo t;
    ThermoF tf;
};

constexpr int kStagedRounds = 15;  // a fast solve takes at most 14 FP64 growth evaluations
constexpr int kStagedListRounds = 3;  // rounds over compacted lists before the finishing launch
// the automatic choice of the staged chain: domains of at least 2^17
// super-droplets (measured on GB300: below that the fused kernel's single
// launch wins; from it the chain, by 10-20 % in 3D)
constexpr int64_t kStagedMinSd = int64_t(1) << 17;
// the rounds over lists of domains of at least 2^22 super-droplets regroup
// tiles of 1024 records (4 per thread); smaller lists keep 256, enough
// blocks to fill the SMs
constexpr int64_t kStagedWideTileSd = int64_t(1) << 22;

__global__ void k_cs_cells(const double *th, const double *rv, const double *rhod, int n_cells, double RH_max,
                           StagedCell *out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const Thermo t = thermo_cond(th[c], rv[c], rhod[c], RH_max, rhod_factor(rhod[c]));
    out[c].t = t;
    out[c].tf = to_float(t);
}

// one warp per cell: every super-droplet's FP32 start, from x0src, r_w^2 at
// the substep's start (the state's at the first substep, then x1)
// The records go to one list of n slots: those whose first FP64 evaluation
// is g(x0) from the front (count n_g0), those that start their polish from
// the back (count n_pol), so that round 0 runs each kind in warps of its own.
__global__ void __launch_bounds__(128, 7) k_cs_start(SdArrays s, const uint32_t *offset, int n_cells, const StagedCell *cells, double dtp,
                           int physics, StagedRec *rec, double *x1, unsigned *n_g0, unsigned *n_pol,
                           unsigned n_sd, const double *x0src) {
    const int64_t c64 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int c = (int)c64, lane = threadIdx.x & 31;
    const bool live = c64 < n_cells;
    const uint32_t beg = live ? offset[c] : 0, end = live ? offset[c + 1] : 0;
    const ThermoF &tf = cells[live ? c : 0].tf;
    // the cell's super-droplets in rounds of 32 (a warp is one cell, so every
    // lane takes the same trips and takes part in the ballots)
    for (uint32_t i0 = beg; i0 < end; i0 += 32) {
        const uint32_t i = i0 + lane;
        int task = kTaskNone;
        FastSolve S;
        if (i < end) {
            const double x0 = x0src[i];
            if (s.N[i] == 0) {
                x1[i] = x0;
            } else {
                S.x0 = x0;
                S.rd3 = s.rd3[i];
                S.kappa = s.kappa[i];
                const int st = fs_start<true>(S, tf, dtp, physics);
                task = cs_task_of(st);
            }
        }
        const unsigned mg = __ballot_sync(0xffffffffu, task != kTaskNone && task != kTaskPolish);
        const unsigned mp = __ballot_sync(0xffffffffu, task == kTaskPolish);
        unsigned bg = 0, bp = 0;
        if (lane == 0) {
            if (mg) bg = atomicAdd(n_g0, (unsigned)__popc(mg));
            if (mp) bp = atomicAdd(n_pol, (unsigned)__popc(mp));
        }
        bg = __shfl_sync(0xffffffffu, bg, 0);
        bp = __shfl_sync(0xffffffffu, bp, 0);
        const unsigned below = (1u << lane) - 1u;
        if (task != kTaskNone) {
            const unsigned pos = task == kTaskPolish ? n_sd - 1u - (bp + __popc(mp & below)) : bg + __popc(mg & below);
            StagedRec &r = rec[pos];
            r.sd = i;
            r.task = task;
            r.S = S;
        }
    }
}

// one FP64 growth evaluation per record; the records that need another go
// to the next list (one atomic per block), the finished write r_w^2.
// FINISH: the last round, each record's evaluations in sequence until its
// solve finishes (the few left after the first rounds)
// Which branches of growth_eval<true> an evaluation at x takes (FP32
// estimate): 0 the Kelvin factor by exp (A/r > 1/32) and the ventilation
// corrections in FP32 (LITE), 1 the same with the Kelvin factor's series,
// 2 the corrections' binomial series, 3 the cube roots, 4 the cube roots and
// Re^0.077 (Re > 1).
SDM_HD int vent_class(float x, const ThermoF &tf, int physics) {
    using namespace phys;
    const float r = sqrtf(x);
    const int kel = tf.A > 0.03125f * r ? 0 : 1;
    if (!physics) return kel;
    const float r3 = x * r;
    const float e = (float)(4.0 / (delta0 * delta0 * sqrt(C0))) * sqrtf(tf.cX * r3);
    const float sq = e / (sqrtf(1.0f + e) + 1.0f);
    const float Re = (float)(delta0 * delta0 / 4.0) * sq * sq, y = Re * fmaxf(tf.Sc, tf.Pr);
    return y <= 5.9604645e-8f ? kel : y <= 0.015625f ? 2 : Re <= 1.0f ? 3 : 4;
}

// RPT records per thread: the regrouping sorts tiles of 256 x RPT records,
// so that fewer warps straddle two classes (for the long lists of large
// domains).
template <bool FINISH, int RPT = 1>
__global__ void __launch_bounds__(256) k_cs_eval(const StagedRec *in, const unsigned *n_in, int64_t rev_end,
                                                 StagedRec *out, unsigned *n_out, const uint32_t *cell_of_sd,
                                                 const StagedCell *cells, double dtp, int physics, double *x1,
                                                 DevStats *st) {
    constexpr int kKeys = 17;  // 3 kinds of record x 5 classes of evaluation, the deferred ends, the empty slots
    constexpr unsigned kTile = 256 * RPT;  // blockDim.x == 256
    __shared__ unsigned s_warp[8], s_base, s_cnt[kKeys];
    __shared__ uint16_t s_perm[kTile];
    const unsigned n = *n_in;
    SolveCounters cnt{0, 0, 0, 0};
    bool bad = false;
    for (unsigned base = blockIdx.x * kTile; base < n; base += gridDim.x * kTile) {
        // the tile's records regrouped by what their round takes (the
        // record's kind, then the branches of growth_eval), so that the lanes
        // of a warp run the same code; each record's arithmetic is unchanged
        int key[RPT];
        unsigned rank[RPT];
        if (threadIdx.x < kKeys) s_cnt[threadIdx.x] = 0;
        __syncthreads();
#pragma unroll
        for (int jj = 0; jj < RPT; ++jj) {
            const unsigned t = base + jj * 256 + threadIdx.x;
            key[jj] = kKeys - 1;
            if (t < n) {
                const StagedRec &q = rev_end ? in[rev_end - 1 - t] : in[t];
                if (q.task == kTaskG0End) {
                    key[jj] = 15;
                } else if (q.task != kTaskNone) {
                    const bool g0 = q.task != kTaskPolish;
                    const int kind = !g0 ? 0 : q.task == kTaskG0Exact ? 1 : 2;
                    key[jj] = 5 * kind + vent_class((float)(g0 ? q.S.x0 : q.S.xk), cells[cell_of_sd[q.sd]].tf, physics);
                }
            }
            rank[jj] = atomicAdd(&s_cnt[key[jj]], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned tot = 0;
            for (int q = 0; q < kKeys; ++q) {
                const unsigned v = s_cnt[q];
                s_cnt[q] = tot;
                tot += v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int jj = 0; jj < RPT; ++jj) s_perm[s_cnt[key[jj]] + rank[jj]] = (uint16_t)(jj * 256 + threadIdx.x);
        __syncthreads();
      for (int jj = 0; jj < RPT; ++jj) {
        const unsigned t = base + s_perm[jj * 256 + threadIdx.x];
        bool keep = false;
        StagedRec r;
        if (t < n) {
            r = rev_end ? in[rev_end - 1 - t] : in[t];  // rev_end: records stored from the back
            if (r.task != kTaskNone) {
                const StagedCell &cl = cells[cell_of_sd[r.sd]];
                FastSolve &S = r.S;
                bool done = false;
                for (int k = 0; k < (FINISH ? kStagedRounds : 1) && !done; ++k)
                    done = cs_step(r.task, S, cl.t, cl.tf, dtp, physics, cnt);
                if (done) {
                    x1[r.sd] = S.x1;
                    bad |= !isfinite(S.x1);
                } else if (FINISH) {
                    // not reached: a fast solve takes at most kStagedRounds - 1
                    // evaluations; flagged rather than left unwritten
                    x1[r.sd] = S.x0;
                    bad = true;
                } else {
                    keep = true;
                }
            }
        }
        if (FINISH) continue;
        // block-wide compaction of the records that continue
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) s_warp[w] = __popc(m);
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned tot = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
                const unsigned v = s_warp[q];
                s_warp[q] = tot;
                tot += v;
            }
            s_base = tot ? atomicAdd(n_out, tot) : 0u;
        }
        __syncthreads();
        if (keep) out[s_base + s_warp[w] + __popc(m & ((1u << lane) - 1u))] = r;
        __syncthreads();
      }
    }
    const unsigned ne = __reduce_add_sync(0xffffffffu, (unsigned)cnt.euler);
    const unsigned nf = __reduce_add_sync(0xffffffffu, (unsigned)cnt.fallback);
    const unsigned anybad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        if (ne) atomicAdd(&st->n_euler, (unsigned long long)ne);
        if (nf) atomicAdd(&st->n_fallback, (unsigned long long)nf);
        if (anybad) atomicOr(&st->flags, kFlagNumeric);
    }
}

// one warp per cell: eq. rhov_update with the new radii, in a fixed order.
// r3[i] holds r_w^3 = x sqrt(x) of the super-droplet's current r_w^2 (set by
// k_cs_cellmap, then by each update for the next substep), so each substep
// takes one square root per super-droplet; fac[c] = -4 pi rho_w / (3 dV
// rho_d), fixed through the call.
__global__ void k_cs_update(SdArrays s, const uint32_t *offset, int n_cells, const StagedCell *cells,
                            const double *x1, double *r3, const double *fac, double *th, double *rv,
                            DevStats *st, bool last) {
    const int64_t c64 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (c64 >= n_cells) return;
    const int c = (int)c64, lane = threadIdx.x & 31;
    double sum = 0.0;
    for (uint32_t i = offset[c] + lane; i < offset[c + 1]; i += 32) {
        const unsigned long long N = s.N[i];
        const double xn = x1[i], r3n = xn * sqrt(xn);
        if (N != 0) sum += (double)N * (r3n - r3[i]);
        r3[i] = r3n;
        if (last) s.rw2[i] = xn;  // earlier substeps' r_w^2 stay in x1, where the next start reads them
    }
    sum = warp_sum(sum);
    if (lane == 0) {
        const Thermo &t = cells[c].t;
        const double drv = fac[c] * sum;
        const double rvn = t.rv + drv, thn = t.th + drv * t.dth_drv;
        rv[c] = rvn;
        th[c] = thn;
        if (!isfinite(rvn) || !isfinite(thn)) atomicOr(&st->flags, kFlagNumeric);
    }
}

// once per call: the cell of every super-droplet, its r_w^3, and each
// cell's factor of eq. rhov_update
__global__ void k_cs_cellmap(SdArrays s, const uint32_t *offset, int n_cells, const double *rhod, double dV,
                             uint32_t *cell_of_sd, double *r3, double *fac) {
    const int64_t c64 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (c64 >= n_cells) return;
    const int c = (int)c64;
    for (uint32_t i = offset[c] + (threadIdx.x & 31); i < offset[c + 1]; i += 32) {
        cell_of_sd[i] = (uint32_t)c;
        const double x0 = s.rw2[i];
        r3[i] = x0 * sqrt(x0);
    }
    if ((threadIdx.x & 31) == 0) fac[c] = -4.0 * phys::pi * phys::rho_w / (3.0 * dV * rhod[c]);
}

static cudaError_t launch_condense_staged(sdm_ctx *c, const sdm_opts &o, int *launches) {
    const int64_t n = c->n_sd;
    const int nc = c->grid.n_cells;
    cudaError_t e = cudaSuccess;
    if (!c->cs_rec[0]) {
        e = cudaMalloc(&c->cs_rec[0], sizeof(StagedRec) * (size_t)n);
        if (e == cudaSuccess) e = cudaMalloc(&c->cs_rec[1], sizeof(StagedRec) * (size_t)n);
        if (e == cudaSuccess) e = cudaMalloc(&c->cs_cell, sizeof(StagedCell) * (size_t)nc + 4 * (size_t)n);
        if (e == cudaSuccess) e = cudaMalloc(&c->cs_x1, 16 * (size_t)n + 8 * (size_t)nc);  // x1, r_w^3, factors
        if (e == cudaSuccess) e = cudaMalloc(&c->cs_cnt, 4 * (kStagedListRounds + 3));
        if (e != cudaSuccess) return e;
    }
    StagedRec *rec[2] = {(StagedRec *)c->cs_rec[0], (StagedRec *)c->cs_rec[1]};
    StagedCell *cells = (StagedCell *)c->cs_cell;
    uint32_t *cell_of_sd = (uint32_t *)(cells + nc);
    const double dtp = c->grid.dt / o.sstp_cond;
    const int64_t warps_threads = (int64_t)nc * 32;
    const int B = 128;
    double *r3 = c->cs_x1 + n, *fac = r3 + n;
    k_cs_cellmap<<<grid_for(warps_threads, B), B, 0, c->stream>>>(c->buf[c->cur], c->offset, nc, c->rhod,
                                                                 c->grid.dV, cell_of_sd, r3, fac);
    *launches = 1 + o.sstp_cond * (kStagedListRounds + 5);  // cells, start, 2 + (rounds - 1) + 1 evals, update
    int dev = 0, n_sm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int eval_blocks = n_sm * 8;
    for (int sub = 0; sub < o.sstp_cond; ++sub) {
        k_cs_cells<<<grid_for(nc, 128), 128, 0, c->stream>>>(c->th, c->rv, c->rhod, nc, o.RH_max, cells);
        // round 0 in two launches, the g(x0) records (front of the list) and
        // the polish records (back); each round's survivors feed the next
        unsigned *cnt = c->cs_cnt, *n_pol = c->cs_cnt + kStagedListRounds + 2;
        e = cudaMemsetAsync(cnt, 0, 4 * (kStagedListRounds + 3), c->stream);
        if (e != cudaSuccess) return e;
        k_cs_start<<<grid_for(warps_threads, B), B, 0, c->stream>>>(c->buf[c->cur], c->offset, nc, cells, dtp,
                                                                   c->oi.physics, rec[0], c->cs_x1, cnt, n_pol,
                                                                   (unsigned)n, sub ? c->cs_x1 : c->buf[c->cur].rw2);
        // round 0 regroups tiles of 1024 records where the lists are long
        for (int part = 0; part < 2; ++part) {
            if (n >= kStagedWideTileSd)
                k_cs_eval<false, 4><<<eval_blocks, 256, 0, c->stream>>>(rec[0], part ? n_pol : cnt, part ? n : 0,
                                                                        rec[1], cnt + 1, cell_of_sd, cells, dtp,
                                                                        c->oi.physics, c->cs_x1, c->dstats);
            else
                k_cs_eval<false><<<eval_blocks, 256, 0, c->stream>>>(rec[0], part ? n_pol : cnt, part ? n : 0,
                                                                     rec[1], cnt + 1, cell_of_sd, cells, dtp,
                                                                     c->oi.physics, c->cs_x1, c->dstats);
        }
        for (int r = 1; r < kStagedListRounds; ++r) {
            if (n >= kStagedWideTileSd)
                k_cs_eval<false, 4><<<eval_blocks, 256, 0, c->stream>>>(rec[r & 1], cnt + r, 0, rec[(r + 1) & 1],
                                                                        cnt + r + 1, cell_of_sd, cells, dtp,
                                                                        c->oi.physics, c->cs_x1, c->dstats);
            else
                k_cs_eval<false><<<eval_blocks, 256, 0, c->stream>>>(rec[r & 1], cnt + r, 0, rec[(r + 1) & 1],
                                                                     cnt + r + 1, cell_of_sd, cells, dtp,
                                                                     c->oi.physics, c->cs_x1, c->dstats);
        }
        const int r = kStagedListRounds;
        k_cs_eval<true><<<eval_blocks, 256, 0, c->stream>>>(rec[r & 1], cnt + r, 0, nullptr, nullptr, cell_of_sd,
                                                            cells, dtp, c->oi.physics, c->cs_x1, c->dstats);
        k_cs_update<<<grid_for(warps_threads, B), B, 0, c->stream>>>(c->buf[c->cur], c->offset, nc, cells, c->cs_x1,
                                                                    r3, fac, c->th, c->rv, c->dstats,
                                                                    sub == o.sstp_cond - 1);
    }
    return cudaGetLastError();
}

// Lanes per cell: 4, 8 or 32 (about eight super-droplets per lane), raised
// while the launch has fewer than ~54 warps per SM (152 SMs), since one
// lane's solves run in sequence and the FP64 pipe needs several warps per
// scheduler.  One-warp blocks when cells are few, so that the last wave is
// fine-grained.
cudaError_t launch_condense(sdm_ctx *c, const sdm_opts &o, int *launches) {
    const int64_t per_cell = (int64_t)c->G * c->oi.sd_conc, n_cells = c->grid.n_cells;
    // the staged chain for the fast FP64 solve where chosen (cond_layout), or
    // by default where the domain holds at least kStagedMinSd super-droplets
    const bool fast64 = c->oi.precision != SDM_PRECISION_MIXED && c->oi.cond_solver != SDM_SOLVER_BISECT;
    const bool staged = c->oi.cond_layout == SDM_COND_STAGED ||
                        (c->oi.cond_layout == SDM_COND_AUTO && c->n_sd >= kStagedMinSd);
    if (fast64 && staged) return launch_condense_staged(c, o, launches);
    int lpc = per_cell <= 32 ? 4 : (per_cell <= 64 ? 8 : 32);
    while (lpc < 32 && n_cells * lpc < (int64_t)32 * 8192) lpc = lpc == 4 ? 8 : 32;
    const int B = n_cells * lpc < (int64_t)32 * 32768 ? 32 : 128;
    if (c->oi.precision == SDM_PRECISION_MIXED) *launches = launch_condense_mode<kModeMixed>(c, o, lpc, B);
    else if (c->oi.cond_solver == SDM_SOLVER_BISECT) *launches = launch_condense_mode<kModeBisect>(c, o, lpc, B);
    else *launches = launch_condense_mode<kModeFast>(c, o, lpc, B);
    return cudaGetLastError();
}

}  // namespace sdm
