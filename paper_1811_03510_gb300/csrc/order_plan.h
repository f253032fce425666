// Geometry of the work order's tiles (order.cu), plain host/device C++ so that it can be tested on the
// host: tiles of TW x TH rays of an image of width w (ray y * w + x; the last row may be partial), their
// sizes, their sample positions and the queue position of each of their rays.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define CCS_HD __host__ __device__
#else
#define CCS_HD
#endif

namespace ccs {

constexpr int kOrderKeys = 16;     // cost classes: candidate patches, clamped to 15
constexpr int kOrderThreads = 256; // threads per block of the estimate and placement kernels

struct OrderGeom {
    uint32_t n, w, h, tiles_x, n_tiles;
};

// Tile shape and samples: TW x TH rays, every SX-th ray in x from SX / 2 and every SY-th in y from SY / 2.
template <int TW_, int TH_, int SX_, int SY_>
struct Shape {
    static constexpr uint32_t TW = TW_, TH = TH_, SX = SX_, SY = SY_;
    static constexpr uint32_t NX = (TW + SX - 1 - SX / 2) / SX, NY = (TH + SY - 1 - SY / 2) / SY;
    static constexpr uint32_t SPT = NX * NY;                  // samples per tile, a divisor of 32
    static constexpr uint32_t TPB = kOrderThreads / SPT;      // tiles per block
    static_assert(32 % SPT == 0, "a tile's samples share a warp");
};
using ImageShape = Shape<8, 8, 4, 4>;
using RunShape = Shape<32, 1, 4, 1>;

// Geometry of n rays in an image of width w (a width beyond the batch is one partial row of n rays).
template <class S>
CCS_HD inline OrderGeom order_geom(uint32_t n, uint32_t w)
{
    OrderGeom g{};
    g.n = n;
    g.w = w < n ? w : n;
    g.h = (uint32_t)(((uint64_t)n + g.w - 1) / g.w);
    g.tiles_x = (g.w + S::TW - 1) / S::TW;
    g.n_tiles = (uint32_t)((uint64_t)g.tiles_x * ((g.h + S::TH - 1) / S::TH));
    return g;
}

template <class S>
CCS_HD inline uint32_t order_blocks(const OrderGeom &g) { return (g.n_tiles + S::TPB - 1) / S::TPB; }

CCS_HD inline uint32_t row_len(const OrderGeom &g, uint32_t y) { return y + 1 < g.h ? g.w : g.n - y * g.w; }

// Rays of the tile at (x0, y0): its rows are full (min(TW, w - x0)) except the image's last row.
template <class S>
CCS_HD inline uint32_t tile_size(const OrderGeom &g, uint32_t x0, uint32_t y0)
{
    const uint32_t row = g.w - x0 < S::TW ? g.w - x0 : S::TW;
    uint32_t s = 0;
#pragma unroll
    for (uint32_t dy = 0; dy < S::TH; ++dy) {
        const uint32_t y = y0 + dy;
        if (y < g.h) {
            const uint32_t len = row_len(g, y);
            s += x0 >= len ? 0u : (len - x0 < row ? len - x0 : row);
        }
    }
    return s;
}

// Sample smp of tile t: its ray index in *j, false where the sample lies outside the image.
template <class S>
CCS_HD inline bool tile_sample(const OrderGeom &g, uint32_t t, uint32_t smp, uint32_t *j)
{
    const uint32_t x = (t % g.tiles_x) * S::TW + S::SX / 2 + (smp % S::NX) * S::SX;
    const uint32_t y = (t / g.tiles_x) * S::TH + S::SY / 2 + (smp / S::NX) * S::SY;
    if (y >= g.h || x >= row_len(g, y)) return false;
    *j = y * g.w + x;
    return true;
}

// Entry e (row-major over TW x TH) of the tile whose first ray sits at (x0, y0): its ray index in *j and
// its offset from the tile's first queue position in *off, false where it lies outside the image.  Only
// the image's last row can be partial, and it is the last row of its tiles, so every earlier row of a
// tile holds min(TW, w - x0) rays.
template <class S>
CCS_HD inline bool tile_entry(const OrderGeom &g, uint32_t x0, uint32_t y0, uint32_t e, uint32_t *j, uint32_t *off)
{
    const uint32_t ly = e / S::TW, lx = e % S::TW;
    const uint32_t x = x0 + lx, y = y0 + ly;
    if (y >= g.h || x >= row_len(g, y)) return false;
    const uint32_t row = g.w - x0 < S::TW ? g.w - x0 : S::TW;
    *j = y * g.w + x;
    *off = ly * row + lx;
    return true;
}

}  // namespace ccs
