// Internal declarations shared by the host table builder and the CUDA
// translation unit of libsbiem.
#pragma once
#include <cstdint>
#include <vector>

namespace sbiem {

// Piecewise Chebyshev interpolants of C^T and C^N on s in [0, npieces * h].
// coef[(p * (deg + 1) + k) * 2 + {0: C^T, 1: C^N}].
struct ChebTable {
  double h = 0.5;
  int deg = 16;
  int npieces = 0;
  std::vector<double> coef;
};

// On-chip weight table of the FP32 history sweep: piece width (a power of
// two, so piece indices and offsets are exact in FP32), the span of each
// piece's polynomial in piece widths, and its degree.
constexpr double kGenH = 0.25;
constexpr double kGenSpan = 1.5;
constexpr int kGenDeg = 5;
// Largest s step of a mode whose weights the sweep evaluates on chip (a
// thread's eight consecutive lags then stay on one piece's polynomial).
constexpr double kGenDsBlockMax = kGenH / 16.0;
// The same for blocks of four consecutive lags (modes with ds above
// kGenDsBlockMax and up to this).
constexpr double kGenDsBlock4Max = kGenH / 8.0;

void kernel_values(double s, double r, double* cT, double* cN);
void build_gen_table(double r, double dt, double smax, std::vector<float>& tab, int* npieces, double* max_err);
void build_cheb(double r, double smax, ChebTable* tab);
void build_twiddles(int64_t N, std::vector<double>& tw);

}  // namespace sbiem
