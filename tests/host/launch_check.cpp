// Host-side check of the launch splitter (csrc/launch.h, for_kind_runs): a
// block range of a table is cut into runs of equal kernel specialisation,
// adjacent entries of one kind merge, empty entries vanish, and more than
// kMaxKindRuns runs fall back to one launch of the dispatching kernel; and
// the kind order of a block table (kind_order): the identity within that
// limit, else a stable sort by kind.
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
  const int nk = kMaxKindRuns + 2;
  std::vector<int> p2(nk + 1), k2(nk);
  for (int i = 0; i <= nk; ++i) p2[i] = 3 * i;
  for (int i = 0; i < nk; ++i) k2[i] = 1 + i % 2;
  const KindTable t2{p2.data(), k2.data(), nk};
  std::vector<Run> most;
  for (int i = 0; i < kMaxKindRuns; ++i) most.push_back({1 + i % 2, 3 * i, 3 * i + 3});
  expect("kMaxKindRuns runs", runs(t2, 0, 3 * kMaxKindRuns), most);
  expect("one run more -> dispatching kernel", runs(t2, 0, 3 * kMaxKindRuns + 3),
         {{kKindGeneral, 0, 3 * kMaxKindRuns + 3}});
  expect("partial first and last", runs(t2, 1, 8), {{1, 1, 3}, {2, 3, 6}, {1, 6, 8}});

  // kind_order: within the limit the identity; beyond it a stable sort, after
  // which the table has one run per kind
  std::vector<int> ord(nk);
  if (kind_order(k2.data(), kMaxKindRuns, ord.data())) {
    std::printf("kind_order sorted a table within the limit\n");
    return 1;
  }
  for (int i = 0; i < kMaxKindRuns; ++i)
    if (ord[i] != i) {
      std::printf("kind_order: not the identity at %d\n", i);
      return 1;
    }
  if (!kind_order(k2.data(), nk, ord.data())) {
    std::printf("kind_order kept %d alternating kinds\n", nk);
    return 1;
  }
  for (int i = 0; i < nk; ++i) {
    const int want = i < nk / 2 ? 2 * i : 2 * (i - nk / 2) + 1;  // kind 1 items, then kind 2, each in order
    if (ord[i] != want) {
      std::printf("kind_order: position %d holds %d, want %d\n", i, ord[i], want);
      return 1;
    }
  }
  std::vector<int> p3(nk + 1, 0), k3(nk);
  for (int i = 0; i < nk; ++i) {
    p3[i + 1] = p3[i] + (p2[ord[i] + 1] - p2[ord[i]]);
    k3[i] = k2[ord[i]];
  }
  const KindTable t3{p3.data(), k3.data(), nk};
  expect("sorted table: one run per kind", runs(t3, 0, 3 * nk), {{1, 0, 3 * nk / 2}, {2, 3 * nk / 2, 3 * nk}});

  // no kind table: the dispatching kernel over the range
  const KindTable none{pre, nullptr, 4};
  expect("no kinds", runs(none, 3, 33), {{kKindGeneral, 3, 33}});

  // the kind <-> length maps of the compile-time kernels
  for (int i = 0; i < kCtLengths; ++i)
    if (ct_index(ct_len(i)) != i || !ct_supported(ct_len(i))) {
      std::printf("ct_len/ct_index differ at %d\n", i);
      return 1;
    }
  if (ct_index(3072) != -1 || ct_supported(2048) || !ct_supported(1024)) {
    std::printf("3072 and 2048 have no compile-time kernel, 1024 has one\n");
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
