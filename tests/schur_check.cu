// Host-side check of the library's per-node Hessenberg / real Schur routines.
// Reads a count and then that many row-major matrices from stdin; prints for
// each the ok flag, then T, then Z (row-major).
//   schur_check           6 x 6, Householder + FP64 Francis iteration
//   schur_check eigvec    5 x 5, the FP32-seeded eigenvector basis
//   schur_check francis32 5 x 5, Householder + FP32 Francis iteration
#include <cstdio>
#include <cstring>

#include "../paper_2404_01407_gb300/csrc/schur.cuh"

template <int BS, typename R>
static void put(bool ok, const R (&T)[BS][BS], const R (&Z)[BS][BS]) {
  printf("%d", ok ? 1 : 0);
  for (int r = 0; r < BS; ++r)
    for (int c = 0; c < BS; ++c) printf(" %.17g", (double)T[r][c]);
  for (int r = 0; r < BS; ++r)
    for (int c = 0; c < BS; ++c) printf(" %.17g", (double)Z[r][c]);
  printf("\n");
}

int main(int argc, char** argv) {
  const char* mode = argc > 1 ? argv[1] : "francis";
  int count = 0;
  if (scanf("%d", &count) != 1) return 1;
  for (int m = 0; m < count; ++m) {
    if (!strcmp(mode, "francis")) {
      double P[6][6], Z[6][6];
      for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) {
          if (scanf("%lf", &P[r][c]) != 1) return 1;
          Z[r][c] = (r == c) ? 1.0 : 0.0;
        }
      fnlh::hessenberg_reduce<6>(P, Z);
      const bool ok = fnlh::schur_real<6>(P, Z);
      put<6>(ok, P, Z);
    } else {
      double A[5][5];
      for (int r = 0; r < 5; ++r)
        for (int c = 0; c < 5; ++c)
          if (scanf("%lf", &A[r][c]) != 1) return 1;
      if (!strcmp(mode, "eigvec")) {
        double Q[5][5], T[5][5];
        const bool ok = fnlh::schur_eigvec<5>(A, Q, T);
        put<5>(ok, T, Q);
      } else {
        float H[5][5], Z[5][5];
        for (int r = 0; r < 5; ++r)
          for (int c = 0; c < 5; ++c) {
            H[r][c] = (float)A[r][c];
            Z[r][c] = (r == c) ? 1.0f : 0.0f;
          }
        fnlh::hessenberg_reduce<5>(H, Z);
        const bool ok = fnlh::schur_real<5>(H, Z);
        put<5>(ok, H, Z);
      }
    }
  }
  return 0;
}
