// CPU driver for the serving loop's admission policy (csrc/admission.h):
// reads scenarios from stdin, prints the admitted ids and what stays queued.
// Input per scenario: n free max_batch, then n lines "kind bytes".
#include <cstdio>
#include <deque>
#include <vector>

#include "admission.h"

struct R { int id, kind; size_t bytes; };

int main() {
  int n, max_batch;
  unsigned long long free_bytes;
  while (std::scanf("%d %llu %d", &n, &free_bytes, &max_batch) == 3) {
    std::vector<R> rs(n);
    std::deque<R*> q;
    for (int i = 0; i < n; ++i) {
      unsigned long long b;
      std::scanf("%d %llu", &rs[i].kind, &b);
      rs[i].id = i;
      rs[i].bytes = (size_t)b;
      q.push_back(&rs[i]);
    }
    size_t taken = 0;
    std::vector<R*> batch = fock::admit_batch(
        q, [](const R* r) { return r->kind != 0; }, [](const R* r) { return r->bytes; },
        (size_t)free_bytes, max_batch, &taken);
    std::printf("batch");
    for (R* r : batch) std::printf(" %d", r->id);
    std::printf(" | left");
    for (R* r : q) std::printf(" %d", r->id);
    std::printf(" | %zu\n", taken);
  }
  return 0;
}
