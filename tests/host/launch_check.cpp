// Host-side check of the launch splitter (csrc/launch.h, for_kind_runs): a
// block range of a table is cut into runs of equal kernel specialisation,
// adjacent entries of one kind merge, empty entries vanish, and more than
// kMaxKindRuns runs fall back to one launch of the dispatching kernel.
// Prints "ok" or the first failing case and exits non-zero.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "launch.h"

using namespace sag;

struct Run {
  int kind, b0, b1;
  bool operator==(const Run& o) const { return kind == o.kind && b0 == o.b0 && b1 == o.b1; }
};

static std::vector<Run> runs(const KindTable& t, int b0, int b1) {
  std::vector<Run> r;
  const cudaError_t e = for_kind_runs(t, b0, b1, [&](int k, int a, int z) {
    r.push_back({k, a, z});
    return cudaSuccess;
  });
  if (e != cudaSuccess) r.push_back({-1, -1, -1});
  return r;
}

static void expect(const char* name, const std::vector<Run>& got, const std::vector<Run>& want) {
  if (got == want) return;
  std::printf("%s: got", name);
  for (const Run& x : got) std::printf(" (%d %d %d)", x.kind, x.b0, x.b1);
  std::printf(", want");
  for (const Run& x : want) std::printf(" (%d %d %d)", x.kind, x.b0, x.b1);
  std::printf("\n");
  std::exit(1);
}

int main() {
  // four items, the second empty: [0,10) kind 12, [10,10) kind 5, [10,25) 12, [25,40) 12
  const int pre[] = {0, 10, 10, 25, 40};
  const int kind[] = {12, 5, 12, 12};
  const KindTable t{pre, kind, 4};
  expect("merge", runs(t, 0, 40), {{12, 0, 40}});
  expect("cut", runs(t, 5, 30), {{12, 5, 30}});
  expect("empty range", runs(t, 7, 7), {});

  // kinds 1 2 1 2 ...: every item its own run
  std::vector<int> p2(11), k2(10);
  for (int i = 0; i <= 10; ++i) p2[i] = 3 * i;
  for (int i = 0; i < 10; ++i) k2[i] = 1 + i % 2;
  const KindTable t2{p2.data(), k2.data(), 10};
  std::vector<Run> eight;
  for (int i = 0; i < 8; ++i) eight.push_back({1 + i % 2, 3 * i, 3 * i + 3});
  expect("eight runs", runs(t2, 0, 24), eight);
  expect("nine runs -> dispatching kernel", runs(t2, 0, 27), {{kKindGeneral, 0, 27}});
  expect("partial first and last", runs(t2, 1, 8), {{1, 1, 3}, {2, 3, 6}, {1, 6, 8}});

  // no kind table: the dispatching kernel over the range
  const KindTable none{pre, nullptr, 4};
  expect("no kinds", runs(none, 3, 33), {{kKindGeneral, 3, 33}});

  // the kind <-> length maps of the compile-time kernels
  for (int i = 0; i < kCtLengths; ++i)
    if (ct_index(ct_len(i)) != i || !ct_supported(ct_len(i))) {
      std::printf("ct_len/ct_index differ at %d\n", i);
      return 1;
    }
  if (ct_index(3072) != -1 || ct_supported(1024)) {
    std::printf("3072 and 1024 have no compile-time kernel\n");
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
