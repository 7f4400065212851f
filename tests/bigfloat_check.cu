// Host program over the multi-limb arithmetic of the Cauchy path (bigfloat.cuh): reads
// operations from stdin, one per line,
//     <op> <L> <a: s e m0 .. m(L-1)> [<b: s e m0 .. m(L-1)>]
// with op one of mul, add, sub, recip, d2b (a double, given as its 64-bit pattern, to
// a value), b2d (a value to the nearest double), and prints the result in the same
// form (d2b, recip, mul, add, sub) or as the double's bit pattern (b2d); limbs in hex,
// m0 the most significant.  Driven by tests/test_bigfloat_host.py.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>

#include "bigfloat.cuh"

using namespace perm;

template <int L>
static bool read_big(Big<L>& a) {
  int s, e;
  if (std::scanf("%d %d", &s, &e) != 2) return false;
  a.s = s;
  a.e = e;
  a.z = 1;
  for (int i = 0; i < L; ++i) {
    unsigned long long v;
    if (std::scanf("%llx", &v) != 1) return false;
    a.m[i] = v;
    if (v) a.z = 0;
  }
  return true;
}

template <int L>
static void print_big(const Big<L>& a) {
  std::printf("%d %d %d", a.s, a.e, a.z);
  for (int i = 0; i < L; ++i) std::printf(" %llx", (unsigned long long)a.m[i]);
  std::printf("\n");
}

template <int L>
static bool run(const std::string& op) {
  Big<L> a, b, r;
  if (op == "d2b") {
    unsigned long long bits;
    if (std::scanf("%llx", &bits) != 1) return false;
    double v;
    std::memcpy(&v, &bits, sizeof v);
    big_from_double(r, v);
    print_big(r);
    return true;
  }
  if (!read_big(a)) return false;
  if (op == "b2d") {
    const double v = big_to_double(a);
    unsigned long long bits;
    std::memcpy(&bits, &v, sizeof bits);
    std::printf("%llx\n", bits);
    return true;
  }
  if (op == "recip") {
    big_recip(r, a);
  } else {
    if (!read_big(b)) return false;
    if (op == "mul") big_mul(r, a, b);
    else if (op == "add") big_add(r, a, b, 0);
    else if (op == "sub") big_add(r, a, b, 1);
    else return false;
  }
  print_big(r);
  return true;
}

int main() {
  char opbuf[16];
  int L;
  while (std::scanf("%15s %d", opbuf, &L) == 2) {
    const std::string op(opbuf);
    bool ok = false;
    switch (L) {
      case 2: ok = run<2>(op); break;
      case 4: ok = run<4>(op); break;
      case 7: ok = run<7>(op); break;
      case 16: ok = run<16>(op); break;
      default: ok = false;
    }
    if (!ok) return 1;
  }
  return 0;
}
