// Generator of ace_nu3.inc: the nu = 3 monomial structure of the ACE basis
// (which products A_a A_b A_c of the 48 entries with n <= 2, l <= 3 occur) as
// straight-line CUDA for the lane-per-atom nu = 3 kernel.  The structure depends
// only on the basis, not on the coefficients.  Regenerate after a change of the
// basis enumeration in ace_tables.cpp:
//   nvcc -std=c++17 -I../../include gen_nu3.cpp ace_tables.cpp -o gen_nu3 && ./gen_nu3 > ace_nu3.inc
#include <cstdio>
#include <cstring>

#include "ap_internal.cuh"

int main() {
  ap_config g;
  std::memset(&g, 0, sizeof(g));
  ap::AceTables t;
  ap::build_ace_tables(g, t);
  const size_t n = t.nu3_key.size();
  std::printf("// Generated by gen_nu3.cpp from the basis enumeration of ace_tables.cpp; do not edit.\n");
  std::printf("// nu = 3 monomials coef[t] * A[a] A[b] A[c] over the 48 entries with n <= 2, l <= 3\n");
  std::printf("// (a <= b <= c): kNu3Key[t] = c | b << 6 | a << 12 in ascending order, and\n");
  std::printf("// AP_NU3_BODY, the gradient of their sum grouped by the factor pair (a, b):\n");
  std::printf("//   p = A[a] A[b]; s = sum_c coef A[c]; dA[c] += coef p; dA[a] += s A[b]; dA[b] += s A[a]\n");
  std::printf("// (the product rule, valid for repeated indices).\n");
  std::printf("#define AP_NU3_N %zu\n", n);
  std::printf("static const unsigned int kNu3Key[AP_NU3_N] = {");
  for (size_t k = 0; k < n; ++k) std::printf("%s%s%u", k ? "," : "", (k % 12) ? "" : "\n    ", t.nu3_key[k]);
  std::printf("};\n");
  size_t groups = 0;
  std::printf("#define AP_NU3_BODY \\\n");
  for (size_t k = 0; k < n;) {
    const unsigned a = (t.nu3_key[k] >> 12) & 63u, b = (t.nu3_key[k] >> 6) & 63u;
    std::printf("  NU3_GROUP_BEGIN(%u, %u)", a, b);
    size_t e = k;
    while (e < n && ((t.nu3_key[e] >> 6) & 4095u) == ((t.nu3_key[k] >> 6) & 4095u)) {
      std::printf(" NU3_TERM(%zu, %u)", e, t.nu3_key[e] & 63u);
      ++e;
    }
    std::printf(" NU3_GROUP_END(%u, %u)%s\n", a, b, e < n ? " \\" : "");
    ++groups;
    k = e;
  }
  std::printf("#define AP_NU3_GROUPS %zu\n", groups);
  return 0;
}
