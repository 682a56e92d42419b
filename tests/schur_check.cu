// Host-side check of the library's per-node Hessenberg / real Schur routines.
// Reads matrices (6x6, row-major) from stdin, prints for each:
//   ok flag, then T (36 values), then Z (36 values).
#include <cstdio>

#include "../paper_2404_01407_gb300/csrc/schur.cuh"

int main() {
  int count = 0;
  if (scanf("%d", &count) != 1) return 1;
  for (int m = 0; m < count; ++m) {
    double P[6][6], Z[6][6];
    for (int r = 0; r < 6; ++r)
      for (int c = 0; c < 6; ++c) {
        if (scanf("%lf", &P[r][c]) != 1) return 1;
        Z[r][c] = (r == c) ? 1.0 : 0.0;
      }
    fnlh::hessenberg_reduce<6>(P, Z);
    const bool ok = fnlh::schur_real<6>(P, Z);
    printf("%d", ok ? 1 : 0);
    for (int r = 0; r < 6; ++r)
      for (int c = 0; c < 6; ++c) printf(" %.17g", P[r][c]);
    for (int r = 0; r < 6; ++r)
      for (int c = 0; c < 6; ++c) printf(" %.17g", Z[r][c]);
    printf("\n");
  }
  return 0;
}
