// Host-side checks of two header-only helpers the GPU path relies on (built with nvcc, run on
// the CPU; no device code runs): the tensor-core weight layout is a bijection, and the float32
// form's power-of-two operand scale puts every finite largest magnitude in [2^13, 2^14).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "../../paper_2108_10209_gb300/csrc/f16_split.cuh"
#include "../../paper_2108_10209_gb300/csrc/tc_layout.cuh"

static int fails = 0;
#define CHECK(c, ...)                 \
  do {                                \
    if (!(c)) {                       \
      ++fails;                        \
      if (fails < 20) printf(__VA_ARGS__); \
    }                                 \
  } while (0)

static unsigned bits(float f) {
  unsigned u;
  memcpy(&u, &f, 4);
  return u;
}

int main() {
  const int widths[4] = {32, 64, 128, 256};
  for (int bf16 = 0; bf16 < 2; ++bf16)
    for (int ci : widths)
      for (int co : widths) {
        const n2f::TcCfg f = n2f::tc_cfg(ci, co, bf16);
        const size_t n = (size_t)9 * ci * co;
        std::vector<unsigned char> seen(n, 0);
        for (int r = 0; r < co; ++r)
          for (int tap = 0; tap < 9; ++tap)
            for (int c = 0; c < ci; ++c) {
              const size_t i = n2f::tc_index_cfg(f, ci, r, tap, c);
              CHECK(i < n, "index out of range %zu (cin %d cout %d bf16 %d)\n", i, ci, co, bf16);
              if (i < n) {
                CHECK(!seen[i], "index %zu hit twice (cin %d cout %d bf16 %d)\n", i, ci, co, bf16);
                seen[i] = 1;
              }
            }
        // 16-byte groups hold GE consecutive input channels of one row and tap
        CHECK(n2f::tc_index_cfg(f, ci, 0, 0, 1) == n2f::tc_index_cfg(f, ci, 0, 0, 0) + 1,
              "channels not contiguous within a group\n");
      }
  for (int k = -126; k <= 127; ++k)
    CHECK(n2f::pow2f(k) == std::ldexp(1.0f, k), "pow2f(%d)\n", k);
  CHECK(n2f::f16_scale_exp(0u) == 0, "scale of zero\n");
  std::mt19937 g(7);
  std::uniform_int_distribution<int> ex(-125, 127);
  std::uniform_real_distribution<float> mant(1.0f, 2.0f);
  for (int t = 0; t < 200000; ++t) {
    const float m = std::ldexp(mant(g), ex(g) - 1);
    if (!std::isfinite(m) || m == 0.f) continue;
    const int k = n2f::f16_scale_exp(bits(m));
    const double s = std::ldexp((double)m, k);
    if (k > -126 && k < 126) {
      CHECK(s >= 8192.0 && s < 16384.0, "m %g k %d scaled %g\n", m, k, s);
    } else {
      CHECK(s < 16384.0, "clamped m %g k %d scaled %g\n", m, k, s);
    }
  }
  // subnormal largest magnitude: clamped scale, still below 2^14
  const float sub = std::ldexp(1.0f, -140);
  CHECK(std::ldexp((double)sub, n2f::f16_scale_exp(bits(sub))) < 16384.0, "subnormal\n");
  printf("%s (%d failures)\n", fails ? "FAIL" : "OK", fails);
  return fails ? 1 : 0;
}
