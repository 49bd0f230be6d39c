// dense_sched.cuh -- the schedule of the deterministic dense assembly,
// shared by its kernels and host code and by a host-side check (plain C++).
//
// Triangles are coloured greedily so that no two triangles of one colour
// share a vertex; the unordered far pairs are then visited colour pair by
// colour pair.  Within one colour (ca == cb) the pairs i < k of the colour's
// list of n triangles are enumerated by a folded triangular grid: block row f
// (0 <= f < (n + 1) / 2) takes the n - 1 - f pairs of row f followed by the
// f pairs of row n - 1 - f, n - 1 pairs in all.
#pragma once

#include <vector>

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

// Pair j (0 <= j < n - 1) of block row f of the folded enumeration of one
// colour list: its positions i < k, or false when (f, j) is past the end.
__host__ __device__ __forceinline__ bool dense_diag_pair(int f, long long j, int n, int *i_out, int *k_out) {
    int i = -1, k = -1;
    if (j < n - 1 - f) {
        i = f;
        k = f + 1 + (int)j;
    } else if (n - 1 - f != f && j < n - 1) {
        i = n - 1 - f;
        k = i + 1 + (int)(j - (n - 1 - f));
    }
    if (i < 0 || k >= n) return false;
    *i_out = i;
    *k_out = k;
    return true;
}

// Greedy colouring in triangle order: col[t] is the smallest colour not used
// by an earlier triangle that shares a vertex with t.  vt_ptr / vt_idx: the
// corners (3 t + a) incident to each vertex.  Returns the number of colours.
inline int dense_colour(int nt, const int *tris, const int *vt_ptr, const int *vt_idx, std::vector<int> &col) {
    col.assign(nt, -1);
    int ncol = 0;
    std::vector<int> seen(64, -1);
    for (int t = 0; t < nt; ++t) {
        for (int a = 0; a < 3; ++a) {
            const int v = tris[3 * t + a];
            for (int e = vt_ptr[v]; e < vt_ptr[v + 1]; ++e) {
                const int c2 = col[vt_idx[e] / 3];
                if (c2 >= 0) {
                    if (c2 >= (int)seen.size()) seen.resize(2 * c2 + 2, -1);
                    seen[c2] = t;
                }
            }
        }
        int c = 0;
        while (c < (int)seen.size() && seen[c] == t) ++c;
        col[t] = c;
        if (c >= (int)seen.size()) seen.resize(2 * c + 2, -1);
        if (c + 1 > ncol) ncol = c + 1;
    }
    return ncol;
}
