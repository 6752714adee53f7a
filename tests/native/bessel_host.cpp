// Host build of the device K_nu quadrature and general-nu Matern correlation
// (bessel.cuh is written for host and device), so that the CPU test-suite can
// check them against an independent implementation of K_nu.
#include "../../paper_2504_12004_gb300/csrc/bessel.cuh"

extern "C" double sbv_test_bessel_k(double nu, double x) { return sbv::bessel_k_trap(nu, x); }
extern "C" double sbv_test_matern_general(double r, double nu) {
  return sbv::matern_general(r, nu);
}
