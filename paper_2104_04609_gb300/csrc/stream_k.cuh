// stream_k.cuh -- the work split of the stream-K tensor-core GEMM, shared by
// its kernels and by a host-side check (plain C++, no CUDA needed).
//
// The product has `tiles` row tiles of KB K slices each: iters = tiles x KB
// iterations, numbered tile-major.  CTA c of G owns the contiguous range
// [c iters / G, (c + 1) iters / G).  Cut at tile boundaries, a range is a
// sequence of segments (one per tile it touches); only its first and last
// segment can cover part of a tile, every segment between them is a whole
// tile.  A whole-tile segment writes C directly; a partial one writes its
// piece to workspace slot 2c (first segment of CTA c) or 2c + 1 (last), and
// the pieces of a tile are summed in CTA order.
#pragma once

#ifndef __CUDACC__
#ifndef __host__
#define __host__
#endif
#ifndef __device__
#define __device__
#endif
#ifndef __forceinline__
#define __forceinline__ inline
#endif
#endif

struct SkSeg {
    int tile, kb0, n;  // K slices kb0 .. kb0 + n - 1 of tile `tile`
};

// First iteration owned by CTA c (c = G gives the end of the last range).
__host__ __device__ __forceinline__ long long sk_begin(int c, long long iters, int G) {
    return (long long)c * iters / G;
}

// The segment that starts at iteration it of a range ending at end.
__host__ __device__ __forceinline__ SkSeg sk_next(long long it, long long end, int KB) {
    SkSeg s;
    s.tile = (int)(it / KB);
    s.kb0 = (int)(it - (long long)s.tile * KB);
    const long long left = end - it;
    s.n = (int)((long long)(KB - s.kb0) < left ? (long long)(KB - s.kb0) : left);
    return s;
}

// Workspace slot of the piece written by segment `seg` (0-based) of CTA c.
__host__ __device__ __forceinline__ int sk_slot(int c, int seg) { return 2 * c + (seg == 0 ? 0 : 1); }

// The CTAs whose ranges meet tile t: c_lo owns its first iteration, c_hi its
// last (s_c <= x  <=>  c <= ceil((x + 1) G / iters) - 1).
__host__ __device__ __forceinline__ void sk_tile_ctas(int tile, int KB, long long iters, int G, int *c_lo,
                                                      int *c_hi) {
    const long long x0 = (long long)tile * KB, x1 = x0 + KB - 1;
    *c_lo = (int)(((x0 + 1) * G + iters - 1) / iters - 1);
    *c_hi = (int)(((x1 + 1) * G + iters - 1) / iters - 1);
}

// Slot holding CTA c's piece of tile t (c_lo <= c <= c_hi, c_lo < c_hi):
// the first segment of c if t is the tile its range starts in, else its last.
__host__ __device__ __forceinline__ int sk_piece_slot(int c, int tile, int KB, long long iters, int G) {
    return 2 * c + ((int)(sk_begin(c, iters, G) / KB) == tile ? 0 : 1);
}
