// Chunk plan of the host-buffer paths (ccs_intersect_host, ccs_intersect_host_batches), plain host C++ so
// that it can be tested on its own: boundaries cut[0..chunks] of at most 8 chunks over n rays, and the
// chunk list of several batches in a row.
#pragma once
#include <stddef.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

namespace ccs {

constexpr uint32_t kHostMaxChunks = 8;

// Given host_chunk: equal chunks of about that size.  Default (host_chunk = 0): a short first and last
// chunk (n/8, at most 2^18 rays), so that little copy time is exposed before the first launch and after
// the last one, and middle chunks of about 2^20 rays; below 2^17 rays, one chunk.  With align > 1 every
// inner boundary is rounded down to a multiple of align (rows of 8-pixel tiles of an image), which can
// leave empty chunks.  Returns the number of chunks.
inline uint32_t host_chunk_plan(uint32_t n, uint32_t host_chunk, size_t align, size_t (&cut)[kHostMaxChunks + 1])
{
    uint32_t chunks;
    if (host_chunk || n < (1u << 17)) {
        const uint64_t per = host_chunk ? host_chunk : (n ? (uint64_t)n : 1);
        chunks = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(kHostMaxChunks, ((uint64_t)n + per - 1) / per));
        for (uint32_t k = 0; k <= chunks; ++k) cut[k] = (size_t)n * k / chunks;
    } else {
        const size_t ramp = std::min<size_t>(n / 8, 1u << 18), middle = n - 2 * ramp;
        const uint32_t mid =
            (uint32_t)std::min<size_t>(kHostMaxChunks - 2, std::max<size_t>(1, (middle + (1u << 20) - 1) >> 20));
        chunks = mid + 2;
        cut[0] = 0;
        for (uint32_t k = 0; k <= mid; ++k) cut[k + 1] = ramp + middle * k / mid;
        cut[chunks] = n;
    }
    if (align > 1)
        for (uint32_t k = 1; k < chunks; ++k) cut[k] = cut[k] / align * align;
    return chunks;
}

// One chunk of a pipeline over several batches: rays [a, a + m) of batch j.
struct HostChunk {
    uint32_t j;
    size_t a, m;
};

// The chunks of batches 0..nb-1 in order, each batch planned by host_chunk_plan with its own chunk size
// and alignment; empty chunks (and so empty batches) are left out.
inline std::vector<HostChunk> host_batch_chunks(uint32_t nb, const uint32_t *n, const uint32_t *host_chunk,
                                                const size_t *align)
{
    std::vector<HostChunk> out;
    for (uint32_t j = 0; j < nb; ++j) {
        if (n[j] == 0) continue;
        size_t cut[kHostMaxChunks + 1];
        const uint32_t c = host_chunk_plan(n[j], host_chunk[j], align[j], cut);
        for (uint32_t k = 0; k < c; ++k)
            if (cut[k + 1] > cut[k]) out.push_back(HostChunk{j, cut[k], cut[k + 1] - cut[k]});
    }
    return out;
}

}  // namespace ccs
