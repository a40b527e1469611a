// Host driver for the blossom matcher of the decoder kernel: reads instances
// (k, then k*k pair weights row-major with -1 = absent, then k boundary
// weights) from stdin and prints "total partner_0 ... partner_{k-1}".
#include <cstdio>
#include <vector>

#include "../paper_2511_05719_gb300/csrc/blossom.cuh"

int main() {
  int k;
  while (std::scanf("%d", &k) == 1) {
    std::vector<long long> w((size_t)k * k), wb(k);
    for (auto& x : w)
      if (std::scanf("%lld", &x) != 1) return 1;
    for (auto& x : wb)
      if (std::scanf("%lld", &x) != 1) return 1;
    std::vector<int> partner(k, -3);
    std::vector<long long> scratch(ttn::boundary_matching_scratch_bytes(k) / 8 + 2);
    auto wp = [&](int i, int j) -> int64_t { return w[(size_t)i * k + j]; };
    auto wbf = [&](int i) -> int64_t { return wb[i]; };
    const int64_t tot = ttn::min_matching_boundary(k, wp, wbf, partner.data(), scratch.data());
    std::printf("%lld", (long long)tot);
    for (int i = 0; i < k; ++i) std::printf(" %d", partner[i]);
    std::printf("\n");
  }
  return 0;
}
