// Pixel-sized Gaussian forward render (Sec. 3.1, Supplement A.3): arguments
// and launch entry shared by gauss.cu and the C ABI.
#pragma once

#include "gvs_internal.cuh"

namespace gvs {

constexpr int GS_TILE = 16;        // target tiles of 16 x 16 pixels, one block each
constexpr int GS_SORT_CAP = 2048;  // tile lists up to this length are sorted in shared memory

// Byte layout of the Gaussian-render workspace (256-byte aligned sections):
// per source pixel two float4 records, per target tile a counter and a 64-bit
// list offset, and the (tile, Gaussian) key lists.
struct GaussLayout {
    int W, H, Wt, Ht, tiles_x, tiles_y, max_tiles;
    size_t off_rec, off_count, off_offset, off_keys, n_keys, total;
};

inline GaussLayout gauss_layout(int W, int H, int Wt, int Ht, int max_radius) {
    auto up = [](size_t n) { return (n + 255) / 256 * 256; };
    GaussLayout g;
    g.W = W; g.H = H; g.Wt = Wt; g.Ht = Ht;
    g.tiles_x = (Wt + GS_TILE - 1) / GS_TILE;
    g.tiles_y = (Ht + GS_TILE - 1) / GS_TILE;
    // a box of 2r + 1 pixels meets at most ceil((2r + 1) / 16) + 1 tiles per axis
    const int span = (2 * max_radius + 1 + GS_TILE - 1) / GS_TILE + 1;
    g.max_tiles = span * span;
    const size_t nt = (size_t)g.tiles_x * g.tiles_y;
    size_t o = 0;
    g.off_rec = o; o = up(o + (size_t)W * H * 32);
    g.off_count = o; o = up(o + nt * 4);
    g.off_offset = o; o = up(o + (nt + 1) * 8);
    g.off_keys = o;
    g.n_keys = (size_t)W * H * g.max_tiles;
    o = up(o + g.n_keys * 8);
    g.total = o;
    return g;
}

struct GaussArgs {
    const void *depth;         // [K][H][W] of depth_dtype
    int depth_dtype;
    const uint32_t *rgba;      // [K][H][W] packed RGBA8
    int W, H, Wt, Ht;
    float scale_px;
    int max_radius;
    float in32[5];             // target fx, fy, cx, cy, fy / fx rounded to FP32
    float4 *color;             // [K][Ht][Wt]: premultiplied rgb, opacity
    float *depth_out;          // [K][Ht][Wt]
    char *ws;
    GaussLayout L;
    ViewXform xf[GVS_MAX_VIEWS];
    float f_ratio[GVS_MAX_VIEWS];
};

cudaError_t launch_gauss_splat(const GaussArgs &a, int K, cudaStream_t st);

}  // namespace gvs
