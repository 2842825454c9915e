/*
 * riemann_exact.c -- exact solution of the 1D Euler Riemann problem for a
 * perfect gas, or two perfect gases of different gamma meeting at the contact.
 * TEST INFRASTRUCTURE ONLY: it supplies the analytic reference for the
 * shock-tube checks of the oracle (L1 convergence).
 *
 * Method: Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics",
 * ch. 4.  The star pressure is the root of f(p) = f_L(p) + f_R(p) + (u_R - u_L),
 * where f_K is the shock (Rankine-Hugoniot) branch for p > p_K and the
 * rarefaction (isentropic) branch otherwise.  f is monotone increasing, so
 * the root is found by plain bisection to the last representable digit.
 */
#include "fx_oracle.h"

#include <math.h>

static double fK(double p, double rK, double pK, double g) {
  double cK = sqrt(g * pK / rK);
  if (p > pK) {
    double A = 2.0 / ((g + 1.0) * rK);
    double B = (g - 1.0) / (g + 1.0) * pK;
    return (p - pK) * sqrt(A / (p + B));
  }
  return 2.0 * cK / (g - 1.0) * (pow(p / pK, (g - 1.0) / (2.0 * g)) - 1.0);
}

/* Star state with (possibly) different ratios of specific heats on the two
 * sides (two perfect gases meeting at the contact): each side's wave
 * function uses its own gamma. */
static int star2(const double WL[3], const double WR[3], double gL, double gR, double star[4]) {
  double rL = WL[0], uL = WL[1], pL = WL[2];
  double rR = WR[0], uR = WR[1], pR = WR[2];
  double cL = sqrt(gL * pL / rL), cR = sqrt(gR * pR / rR);
  double du = uR - uL;
  /* pressure positivity condition: no vacuum */
  if (2.0 * cL / (gL - 1.0) + 2.0 * cR / (gR - 1.0) <= du) return -1;
  double lo = 0.0, hi = fmax(pL, pR);
  while (fK(hi, rL, pL, gL) + fK(hi, rR, pR, gR) + du < 0.0) hi *= 2.0;
  for (int it = 0; it < 2000; it++) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (fK(mid, rL, pL, gL) + fK(mid, rR, pR, gR) + du < 0.0) lo = mid;
    else hi = mid;
  }
  double ps = 0.5 * (lo + hi);
  double us = 0.5 * (uL + uR) + 0.5 * (fK(ps, rR, pR, gR) - fK(ps, rL, pL, gL));
  double gmL = (gL - 1.0) / (gL + 1.0), gmR = (gR - 1.0) / (gR + 1.0);
  double rsL = ps > pL ? rL * (ps / pL + gmL) / (gmL * ps / pL + 1.0) : rL * pow(ps / pL, 1.0 / gL);
  double rsR = ps > pR ? rR * (ps / pR + gmR) / (gmR * ps / pR + 1.0) : rR * pow(ps / pR, 1.0 / gR);
  star[0] = ps; star[1] = us; star[2] = rsL; star[3] = rsR;
  return 0;
}

static int sample2(const double WL[3], const double WR[3], double gL, double gR, double xi,
                   double out[3]) {
  double star[4];
  if (star2(WL, WR, gL, gR, star)) return -1;
  double ps = star[0], us = star[1];
  double rL = WL[0], uL = WL[1], pL = WL[2];
  double rR = WR[0], uR = WR[1], pR = WR[2];
  if (xi <= us) {               /* left of the contact */
    double g = gL;
    double cL = sqrt(g * pL / rL);
    double e1 = (g - 1.0) / (2.0 * g), e2 = (g + 1.0) / (2.0 * g);
    if (ps > pL) {              /* left shock */
      double S = uL - cL * sqrt(e2 * ps / pL + e1);
      if (xi <= S) { out[0] = rL; out[1] = uL; out[2] = pL; }
      else { out[0] = star[2]; out[1] = us; out[2] = ps; }
    } else {                    /* left rarefaction */
      double head = uL - cL;
      double csL = cL * pow(ps / pL, e1);
      double tail = us - csL;
      if (xi <= head) { out[0] = rL; out[1] = uL; out[2] = pL; }
      else if (xi > tail) { out[0] = star[2]; out[1] = us; out[2] = ps; }
      else {
        double br = 2.0 / (g + 1.0) + (g - 1.0) / ((g + 1.0) * cL) * (uL - xi);
        out[0] = rL * pow(br, 2.0 / (g - 1.0));
        out[1] = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * uL + xi);
        out[2] = pL * pow(br, 2.0 * g / (g - 1.0));
      }
    }
  } else {                      /* right of the contact */
    double g = gR;
    double cR = sqrt(g * pR / rR);
    double e1 = (g - 1.0) / (2.0 * g), e2 = (g + 1.0) / (2.0 * g);
    if (ps > pR) {              /* right shock */
      double S = uR + cR * sqrt(e2 * ps / pR + e1);
      if (xi >= S) { out[0] = rR; out[1] = uR; out[2] = pR; }
      else { out[0] = star[3]; out[1] = us; out[2] = ps; }
    } else {                    /* right rarefaction */
      double head = uR + cR;
      double csR = cR * pow(ps / pR, e1);
      double tail = us + csR;
      if (xi >= head) { out[0] = rR; out[1] = uR; out[2] = pR; }
      else if (xi <= tail) { out[0] = star[3]; out[1] = us; out[2] = ps; }
      else {
        double br = 2.0 / (g + 1.0) - (g - 1.0) / ((g + 1.0) * cR) * (uR - xi);
        out[0] = rR * pow(br, 2.0 / (g - 1.0));
        out[1] = 2.0 / (g + 1.0) * (-cR + 0.5 * (g - 1.0) * uR + xi);
        out[2] = pR * pow(br, 2.0 * g / (g - 1.0));
      }
    }
  }
  return 0;
}

int or_riemann_star(const double WL[3], const double WR[3], double g, double star[4]) {
  return star2(WL, WR, g, g, star);
}

int or_riemann_sample(const double WL[3], const double WR[3], double g, double xi,
                      double out[3]) {
  return sample2(WL, WR, g, g, xi, out);
}

int or_riemann_star2(const double WL[3], const double WR[3], double gL, double gR,
                     double star[4]) {
  return star2(WL, WR, gL, gR, star);
}

int or_riemann_sample2(const double WL[3], const double WR[3], double gL, double gR, double xi,
                       double out[3]) {
  return sample2(WL, WR, gL, gR, xi, out);
}
