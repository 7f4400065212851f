// Exercises include/permanent.hpp, the C++ interface in the shape of the paper's
// library, against closed forms; prints one line per check and exits non-zero on the
// first failure.  Built and run by tests/test_gpu_paper_api.py.
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <stdexcept>
#include <vector>

#include "permanent.hpp"

static int failures = 0;

static void expect(bool ok, const char* what) {
  std::printf("%s %s\n", ok ? "ok" : "FAIL", what);
  if (!ok) ++failures;
}

int main() {
  // the usage section's example: per = 450
  const int64_t worked[9] = {1, 2, 3, 4, 5, 6, 7, 8, 9};
  expect(permanent::opt(3, 3, worked) == 450.0, "opt<int64_t> returns double 450");
  expect(permanent::glynn<int64_t, int64_t>(3, 3, worked) == 450, "glynn<int64_t, int64_t> exact 450");
  expect(permanent::ryser_square<int64_t, int32_t>(3, 3, worked) == 450, "ryser_square<int64_t, int32_t>");
  expect(permanent::combinatoric<int64_t, __int128>(3, 3, worked) == 450, "combinatoric<.., __int128>");
  const double wd[9] = {1, 2, 3, 4, 5, 6, 7, 8, 9};
  expect(std::fabs(permanent::glynn(3, 3, wd) - 450.0) < 1e-12, "glynn<double>");
  const float wf[9] = {1, 2, 3, 4, 5, 6, 7, 8, 9};
  expect(std::fabs(permanent::ryser(3, 3, wf) - 450.0) < 1e-12, "ryser<float>");
  std::complex<double> wc[9];
  for (int k = 0; k < 9; ++k) wc[k] = std::complex<double>(wd[k], wd[k]);  // (1 + i) A
  const std::complex<double> want = 450.0 * std::pow(std::complex<double>(1, 1), 3);
  expect(std::abs(permanent::opt(3, 3, wc) - want) < 1e-9, "opt<complex<double>>");
  // Gaussian integers, exact: per((1 + i) A) = (1 + i)^3 450 = -900 + 900 i
  std::complex<int64_t> wg[9];
  for (int k = 0; k < 9; ++k) wg[k] = std::complex<int64_t>(worked[k], worked[k]);
  const std::complex<int64_t> g = permanent::glynn<std::complex<int64_t>, int64_t>(3, 3, wg);
  expect(g.real() == -900 && g.imag() == 900, "glynn<complex<int64_t>, int64_t>");
  // rectangular all-ones: n! / (n - m)!; m > n is per(A^T)
  const std::vector<double> ones(2 * 4, 1.0);
  expect(permanent::glynn_rectangular(2, 4, ones.data()) == 12.0, "glynn_rectangular 2x4 ones");
  expect(permanent::ryser(4, 2, ones.data()) == 12.0, "ryser 4x2 ones (transpose)");
  bool threw = false;
  try {
    permanent::opt_square(2, 4, ones.data());
  } catch (const std::invalid_argument&) {
    threw = true;
  }
  expect(threw, "opt_square refuses 2x4");
  // 0/1 input: per(J_n) = n!; 21! does not fit int64
  const std::vector<uint8_t> j21(21 * 21, 1);
  expect(permanent::glynn<uint8_t, __int128>(21, 21, j21.data()) == (__int128)2432902008176640000 * 21,
         "glynn<uint8_t, __int128> 21!");
  threw = false;
  try {
    permanent::glynn<uint8_t, int64_t>(21, 21, j21.data());
  } catch (const std::overflow_error&) {
    threw = true;
  }
  expect(threw, "21! into int64_t throws overflow_error");
  return failures ? 1 : 0;
}
