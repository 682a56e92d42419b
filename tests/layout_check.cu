// Host-side dump of the library's internal vector layout (csrc/common.cuh):
// for b = 5 and 6, K = 1..5 systems and FP32 / FP64 vectors, one line
//   b elem K real_mean node_stride  then per k: sys_offset slice_len
// and for b = 5 and 6 one line
//   b kMeanSlot  mean_pos(0..b-1)  mean_pad(0..kMeanSlot-1)
#include <cstdio>

#include "../paper_2404_01407_gb300/csrc/common.cuh"

template <int BS, typename T>
void dump() {
  for (int K = 1; K <= 5; ++K) {
    printf("S %d %d %d %d %zu", BS, (int)sizeof(T), K, fnlh::real_mean<T>(K) ? 1 : 0, fnlh::node_stride<BS, T>(K));
    for (int k = 0; k < K; ++k) printf(" %zu %d", fnlh::sys_offset<BS, T>(K, k), fnlh::slice_len<BS, T>(K, k));
    printf("\n");
  }
}

template <int BS>
void dump_mean() {
  printf("M %d %d", BS, fnlh::kMeanSlot<BS>);
  for (int t = 0; t < BS; ++t) printf(" %d", fnlh::mean_pos<BS>(t));
  for (int e = 0; e < fnlh::kMeanSlot<BS>; ++e) printf(" %d", fnlh::mean_pad<BS>(e) ? 1 : 0);
  printf("\n");
}

int main() {
  dump<5, float>();
  dump<6, float>();
  dump<5, double>();
  dump<6, double>();
  dump_mean<5>();
  dump_mean<6>();
  return 0;
}
