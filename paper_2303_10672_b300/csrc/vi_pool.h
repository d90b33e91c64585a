// vi_pool.h -- per-process cache of device blocks, pinned host blocks and
// streams used by problem handles (vi_pool.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "../../include/vi.h"

namespace vip {
// a device block of at least `bytes` on the current device (cached or new)
cudaError_t dev_alloc(void **p, size_t bytes);
// a pinned host block of at least `bytes`
cudaError_t host_alloc(void **p, size_t bytes);
// return a block from dev_alloc / host_alloc; no queued work may still use it
void release(void *p);
// a non-blocking stream of the current device, and its return
cudaError_t stream_get(cudaStream_t *s);
void stream_put(cudaStream_t s);
// free every cached block and idle stream; returns the bytes freed
size_t trim();
size_t cached_bytes();

template <typename T>
cudaError_t dev_alloc_t(T **p, size_t bytes) {
    return dev_alloc((void **)p, bytes);
}
}  // namespace vip
