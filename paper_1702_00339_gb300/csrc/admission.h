// Admission policy of the serving loop (host only; no CUDA).
//
// From a FIFO queue of requests, a free worker takes the head request and,
// in queue order, the later requests of the same kind, stopping at the
// first request of that kind that does not fit the free HBM bytes, and at
// the batch cap.  Requests of the other kind keep their places.  The head
// is always considered first, so no request waits for more than the batches
// ahead of it; within a kind the order is FIFO.
#ifndef FOCK_ADMISSION_H
#define FOCK_ADMISSION_H

#include <cstddef>
#include <deque>
#include <vector>

namespace fock {

// Moves the admitted requests from `pending` into the returned batch (queue
// order) and adds their bytes to *taken.  kind_of(r) -> bool, bytes_of(r) ->
// size_t.  An empty batch means the head does not fit `free_bytes`.
template <class T, class KindOf, class BytesOf>
std::vector<T*> admit_batch(std::deque<T*>& pending, KindOf kind_of, BytesOf bytes_of, size_t free_bytes,
                            int max_batch, size_t* taken) {
  std::vector<T*> batch;
  size_t bytes = 0;
  if (pending.empty() || max_batch <= 0) {
    *taken = 0;
    return batch;
  }
  const bool kind = kind_of(pending.front());
  for (auto q = pending.begin(); q != pending.end() && (int)batch.size() < max_batch;) {
    T* r = *q;
    if (kind_of(r) != kind) { ++q; continue; }
    const size_t b = bytes_of(r);
    if (b > free_bytes - bytes) break;   // bytes <= free_bytes holds throughout
    batch.push_back(r);
    bytes += b;
    q = pending.erase(q);
  }
  *taken = bytes;
  return batch;
}

}  // namespace fock

#endif
