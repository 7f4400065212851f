/*
 * permanent.hpp -- header-only C++ interface in the shape of the paper's library
 * (its usage section), over the C ABI of perm.h:
 *
 *     template <typename Type, typename IntType = void>
 *     permanent::result_t<Type, IntType> permanent::fn(size_t m, size_t n, const Type* ptr);
 *
 * with fn one of combinatoric, glynn, ryser, opt (the learned dispatcher, perm_auto),
 * each also with the suffix _square or _rectangular (which check the shape and throw
 * std::invalid_argument otherwise).  `ptr` is an m x n row-major matrix in host
 * memory; m > n is evaluated as per(A^T).
 *
 * Type: double, float, std::complex<double>, std::complex<float>, an integer type
 * (computed exactly in int128: uint8_t / bool as PERM_U8, other integers as int64),
 * or std::complex of a signed integer type (Gaussian integers, exact).
 * result_t<Type, void> is double (std::complex<double> for complex Type); with an
 * integer Type, IntType may name an integer return type (std::complex<IntType> for
 * complex integer Type), filled from the exact result: a value that does not fit
 * throws std::overflow_error.  Errors reported by the library throw
 * std::runtime_error with perm_status_string's text (PERM_EOVERFLOW when an integer
 * result could not be guaranteed exact).
 *
 * Each calling thread lazily creates one handle, on CUDA device 0 unless
 * permanent::set_device chose another before the thread's first call; the calls run
 * on the legacy default stream and return when the result is on the host.  C++17.
 */
#ifndef PERMANENT_HPP_
#define PERMANENT_HPP_

#include <complex>
#include <cstddef>
#include <cstdint>
#include <limits>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <vector>

#include "perm.h"

namespace permanent {

namespace detail {

template <typename T>
struct is_complex : std::false_type {};
template <typename T>
struct is_complex<std::complex<T>> : std::true_type {};
template <typename T>
struct scalar_of {
  using type = T;
};
template <typename T>
struct scalar_of<std::complex<T>> {
  using type = T;
};

template <typename Type, typename IntType, typename = void>
struct result_impl {
  static_assert(std::is_void<IntType>::value, "IntType needs an integer Type");
  using type = typename std::conditional<is_complex<Type>::value, std::complex<double>, double>::type;
};
template <typename Type, typename IntType>
struct result_impl<Type, IntType,
                   typename std::enable_if<!std::is_void<IntType>::value &&
                                           std::is_integral<typename scalar_of<Type>::type>::value>::type> {
  using type = typename std::conditional<is_complex<Type>::value, std::complex<IntType>, IntType>::type;
};

struct Handle {
  perm_handle h = nullptr;
  ~Handle() {
    if (h) perm_destroy(h);
  }
};

inline int& device_choice() {
  thread_local int device = 0;
  return device;
}

inline perm_handle handle() {
  thread_local Handle hd;
  if (!hd.h) {
    const int rc = perm_create(&hd.h, device_choice());
    if (rc != PERM_OK) {
      hd.h = nullptr;
      throw std::runtime_error(std::string("perm_create: ") + perm_status_string(rc));
    }
  }
  return hd.h;
}

using Entry = int (*)(perm_handle, const void*, int64_t, int64_t, int64_t, int, void*, void*, const perm_opts*);

inline void check(int rc, const char* where) {
  if (rc != PERM_OK) throw std::runtime_error(std::string(where) + ": " + perm_status_string(rc));
}

// two's-complement int128 {low, high} -> the value, then into R with a range check
template <typename R>
R from_int128(uint64_t lo, uint64_t hi) {
  const __int128 v = (__int128)(((unsigned __int128)hi << 64) | lo);
  if constexpr (!std::is_floating_point<R>::value) {
    if (v < (__int128)std::numeric_limits<R>::min() || v > (__int128)std::numeric_limits<R>::max())
      throw std::overflow_error("permanent: the exact result does not fit the requested IntType");
  }
  return (R)v;
}

template <typename Type, typename IntType>
typename result_impl<Type, IntType>::type call(Entry fn, const char* name, size_t m, size_t n, const Type* ptr) {
  using Scalar = typename scalar_of<Type>::type;
  using Result = typename result_impl<Type, IntType>::type;
  static_assert(std::is_arithmetic<Scalar>::value, "permanent: unsupported element type");
  const size_t count = m * n;
  perm_handle h = handle();
  if constexpr (std::is_floating_point<Scalar>::value && !is_complex<Type>::value) {
    std::vector<double> a(ptr, ptr + count);
    double out = 0.0;
    check(fn(h, a.data(), (int64_t)m, (int64_t)n, (int64_t)n, PERM_F64, &out, nullptr, nullptr), name);
    return Result(out);
  } else if constexpr (std::is_floating_point<Scalar>::value) {
    std::vector<std::complex<double>> a(count);
    for (size_t k = 0; k < count; ++k) a[k] = std::complex<double>(ptr[k]);
    double out[2] = {0.0, 0.0};
    check(fn(h, a.data(), (int64_t)m, (int64_t)n, (int64_t)n, PERM_C128, out, nullptr, nullptr), name);
    return Result(std::complex<double>(out[0], out[1]));
  } else if constexpr (!is_complex<Type>::value) {
    using R = typename std::conditional<std::is_void<IntType>::value, double, IntType>::type;
    uint64_t out[2] = {0, 0};
    if constexpr (std::is_same<Scalar, bool>::value || std::is_same<Scalar, uint8_t>::value) {
      std::vector<uint8_t> a(count);
      for (size_t k = 0; k < count; ++k) a[k] = (uint8_t)ptr[k];
      check(fn(h, a.data(), (int64_t)m, (int64_t)n, (int64_t)n, PERM_U8, out, nullptr, nullptr), name);
    } else {
      std::vector<int64_t> a(count);
      for (size_t k = 0; k < count; ++k) {
        if (std::is_unsigned<Scalar>::value && (uint64_t)ptr[k] > (uint64_t)std::numeric_limits<int64_t>::max())
          throw std::overflow_error("permanent: an entry does not fit int64");
        a[k] = (int64_t)ptr[k];
      }
      check(fn(h, a.data(), (int64_t)m, (int64_t)n, (int64_t)n, PERM_I64, out, nullptr, nullptr), name);
    }
    return Result(from_int128<R>(out[0], out[1]));
  } else {
    static_assert(std::is_signed<Scalar>::value, "permanent: complex integers must be signed");
    using R = typename std::conditional<std::is_void<IntType>::value, double, IntType>::type;
    std::vector<int64_t> a(2 * count);
    for (size_t k = 0; k < count; ++k) {
      a[2 * k] = (int64_t)ptr[k].real();
      a[2 * k + 1] = (int64_t)ptr[k].imag();
    }
    uint64_t out[4] = {0, 0, 0, 0};
    check(fn(h, a.data(), (int64_t)m, (int64_t)n, (int64_t)n, PERM_CI64, out, nullptr, nullptr), name);
    return Result(std::complex<R>(from_int128<R>(out[0], out[1]), from_int128<R>(out[2], out[3])));
  }
}

inline void check_shape(size_t m, size_t n, int want, const char* name) {
  if (want == 1 && m != n) throw std::invalid_argument(std::string(name) + ": the matrix is not square");
  if (want == 2 && m == n) throw std::invalid_argument(std::string(name) + ": the matrix is square");
}

}  // namespace detail

template <typename Type, typename IntType = void>
using result_t = typename detail::result_impl<Type, IntType>::type;

// Device of the calling thread's handle (takes effect before its first call).
inline void set_device(int device) { detail::device_choice() = device; }

#define PERMANENT_HPP_FUNCTIONS(fn, entry)                                                         \
  template <typename Type, typename IntType = void>                                                \
  result_t<Type, IntType> fn(const size_t m, const size_t n, const Type* ptr) {                    \
    return detail::call<Type, IntType>(entry, #fn, m, n, ptr);                                     \
  }                                                                                                \
  template <typename Type, typename IntType = void>                                                \
  result_t<Type, IntType> fn##_square(const size_t m, const size_t n, const Type* ptr) {           \
    detail::check_shape(m, n, 1, #fn "_square");                                                   \
    return detail::call<Type, IntType>(entry, #fn "_square", m, n, ptr);                           \
  }                                                                                                \
  template <typename Type, typename IntType = void>                                                \
  result_t<Type, IntType> fn##_rectangular(const size_t m, const size_t n, const Type* ptr) {      \
    detail::check_shape(m, n, 2, #fn "_rectangular");                                              \
    return detail::call<Type, IntType>(entry, #fn "_rectangular", m, n, ptr);                      \
  }

PERMANENT_HPP_FUNCTIONS(combinatoric, perm_combinatoric)
PERMANENT_HPP_FUNCTIONS(glynn, perm_glynn)
PERMANENT_HPP_FUNCTIONS(ryser, perm_ryser)
PERMANENT_HPP_FUNCTIONS(opt, perm_auto)

#undef PERMANENT_HPP_FUNCTIONS

}  // namespace permanent

#endif /* PERMANENT_HPP_ */
