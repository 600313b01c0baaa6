// Host check of the request server's grouping policy (test infrastructure):
// group_cap and group_size_for from server_policy.h on fixed cases.
// Prints "ok" and exits 0, or the failing case and exits 1.
#include <cstdio>
#include <stdexcept>

#include "server_policy.h"

using hz::group_cap;
using hz::group_size_for;

static int fails = 0;
static void expect(bool ok, const char* what) {
  if (!ok) {
    printf("FAIL: %s\n", what);
    ++fails;
  }
}

int main() {
  const size_t GB = 1ull << 30;
  // the host staging cap: 1 GiB of complex doubles per group
  expect(group_cap(8, 129 * 129) == 8, "small grid keeps group_max");
  expect(group_cap(64, 2049LL * 2049) == 8, "2049^2: 16 x 16 B x 4.2M > 1 GiB, 8 fits");
  expect(group_cap(64, 193LL * 193 * 193) == 8, "193^3: 8 x 16 B x 7.2M < 1 GiB");
  expect(group_cap(2, 1LL << 40) == 1, "nothing fits: alone");
  auto lin = [](size_t base, size_t per) { return [=](int k) { return base + per * (size_t)k; }; };
  size_t b = 0;
  // powers of two only: 1 + candidates rounded down
  expect(group_size_for(0, 0, 0, GB, lin(100, 10), &b) == 1, "no candidates");
  expect(group_size_for(1, 0, 0, GB, lin(100, 10), &b) == 2 && b == 120, "two");
  expect(group_size_for(2, 0, 0, GB, lin(100, 10), &b) == 2, "three -> two");
  expect(group_size_for(5, 0, 0, GB, lin(100, 10), &b) == 4 && b == 140, "six -> four");
  expect(group_size_for(7, 0, 0, GB, lin(100, 10), &b) == 8 && b == 180, "eight");
  // the budget: the leader's own bytes are replaced by the group's
  expect(group_size_for(7, 1000, 110, 1000 - 110 + 140, lin(100, 10), &b) == 4, "budget allows four");
  expect(group_size_for(7, 1000, 110, 1000 - 110 + 119, lin(100, 10), &b) == 1, "budget allows none");
  expect(group_size_for(7, 1000, 110, 1000 - 110 + 120, lin(100, 10), &b) == 2 && b == 120, "budget allows two");
  // a size the library refuses keeps the request alone
  auto refuse = [](int) -> size_t { throw std::runtime_error("no"); };
  expect(group_size_for(7, 0, 0, GB, refuse, &b) == 1, "refused");
  if (fails) return 1;
  printf("ok\n");
  return 0;
}
