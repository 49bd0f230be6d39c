// Host check of the deterministic dense assembly's schedule (dense_sched.cuh):
//  - the folded enumeration of one colour list (block rows f < (n + 1) / 2,
//    ceil((n - 1) / P) blocks of P pairs each) yields every pair i < k once;
//  - the greedy colouring is proper (triangles sharing a vertex differ) and
//    greedy (every smaller colour is taken by an earlier neighbour);
//  - visiting colour pairs ca <= cb yields every unordered triangle pair once,
//    and within one launch no matrix entry (vertex of the test triangle,
//    vertex of the source triangle) has two writers, counting the reverse
//    orientation that a same-colour launch also writes.
// Prints "ok <cases>" and exits 0, or the first violation and exits 1.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <set>
#include <utility>
#include <vector>

#include "../paper_2104_04609_gb300/csrc/dense_sched.cuh"

static int check_fold(int n, int P) {
    const int gx = (n - 1 + P - 1) / P, gy = (n + 1) / 2;
    std::vector<int> seen((size_t)n * n, 0);
    for (int f = 0; f < gy; ++f)
        for (int bx = 0; bx < gx; ++bx)
            for (int lp = 0; lp < P; ++lp) {
                int i, k;
                if (!dense_diag_pair(f, (long long)bx * P + lp, n, &i, &k)) continue;
                if (i < 0 || k >= n || i >= k) {
                    std::printf("FAIL fold pair out of range n=%d P=%d\n", n, P);
                    return 1;
                }
                ++seen[(size_t)i * n + k];
            }
    for (int i = 0; i < n; ++i)
        for (int k = i + 1; k < n; ++k)
            if (seen[(size_t)i * n + k] != 1) {
                std::printf("FAIL fold pair (%d, %d) seen %d times, n=%d P=%d\n", i, k, seen[(size_t)i * n + k], n,
                            P);
                return 1;
            }
    return 0;
}

struct Mesh {
    int nv;
    std::vector<int> tris, vt_ptr, vt_idx;
};

static void incidence(Mesh &m) {
    const int nt = (int)m.tris.size() / 3;
    m.vt_ptr.assign(m.nv + 1, 0);
    for (int c = 0; c < 3 * nt; ++c) ++m.vt_ptr[m.tris[c] + 1];
    for (int v = 0; v < m.nv; ++v) m.vt_ptr[v + 1] += m.vt_ptr[v];
    m.vt_idx.assign(3 * nt, 0);
    std::vector<int> fill(m.vt_ptr.begin(), m.vt_ptr.end() - 1);
    for (int c = 0; c < 3 * nt; ++c) m.vt_idx[fill[m.tris[c]]++] = c;
}

static Mesh torus(int nx, int ny) {  // closed triangulated torus, 2 nx ny triangles
    Mesh m;
    m.nv = nx * ny;
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j) {
            const int a = i * ny + j, b = ((i + 1) % nx) * ny + j, c = ((i + 1) % nx) * ny + (j + 1) % ny,
                      d = i * ny + (j + 1) % ny;
            m.tris.insert(m.tris.end(), {a, b, c, a, c, d});
        }
    incidence(m);
    return m;
}

static Mesh random_soup(int nv, int nt, unsigned seed) {  // heavy vertex sharing
    Mesh m;
    m.nv = nv;
    std::srand(seed);
    for (int t = 0; t < nt; ++t) {
        int a = std::rand() % nv, b = std::rand() % nv, c = std::rand() % nv;
        while (b == a) b = std::rand() % nv;
        while (c == a || c == b) c = std::rand() % nv;
        m.tris.insert(m.tris.end(), {a, b, c});
    }
    incidence(m);
    return m;
}

static Mesh fan(int k) {  // k triangles around vertex 0: k colours needed
    Mesh m;
    m.nv = k + 1;
    for (int t = 0; t < k; ++t) m.tris.insert(m.tris.end(), {0, 1 + t, 1 + (t + 1) % k});
    incidence(m);
    return m;
}

static int check_mesh(const Mesh &m, const char *name) {
    const int nt = (int)m.tris.size() / 3;
    std::vector<int> col;
    const int ncol = dense_colour(nt, m.tris.data(), m.vt_ptr.data(), m.vt_idx.data(), col);
    auto share = [&](int t, int s) {
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                if (m.tris[3 * t + a] == m.tris[3 * s + b]) return true;
        return false;
    };
    int mx = -1;
    for (int t = 0; t < nt; ++t) {
        if (col[t] < 0 || col[t] >= ncol) {
            std::printf("FAIL %s colour out of range\n", name);
            return 1;
        }
        mx = col[t] > mx ? col[t] : mx;
        std::set<int> nb;
        for (int s = 0; s < t; ++s)
            if (share(t, s)) nb.insert(col[s]);
        for (int s = 0; s < nt; ++s)
            if (s != t && share(t, s) && col[s] == col[t]) {
                std::printf("FAIL %s triangles %d, %d share a vertex and colour %d\n", name, t, s, col[t]);
                return 1;
            }
        for (int c = 0; c < col[t]; ++c)
            if (!nb.count(c)) {
                std::printf("FAIL %s colour of %d not greedy\n", name, t);
                return 1;
            }
    }
    if (mx + 1 != ncol) {
        std::printf("FAIL %s colour count\n", name);
        return 1;
    }
    // colour lists (ascending triangle order) and the launch schedule
    std::vector<std::vector<int>> lists(ncol);
    for (int t = 0; t < nt; ++t) lists[col[t]].push_back(t);
    std::map<std::pair<int, int>, int> pairs;
    for (int ca = 0; ca < ncol; ++ca)
        for (int cb = ca; cb < ncol; ++cb) {
            const std::vector<int> &la = lists[ca], &lb = lists[cb];
            std::map<std::pair<int, int>, int> writers;  // entry (row vertex, column vertex) -> writes
            auto write = [&](int t, int s) {             // test t, source s
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) ++writers[{m.tris[3 * t + a], m.tris[3 * s + b]}];
            };
            if (ca == cb) {
                const int n = (int)la.size();
                if (n < 2) continue;
                const int P = 16, gx = (n - 1 + P - 1) / P, gy = (n + 1) / 2;
                for (int f = 0; f < gy; ++f)
                    for (int bx = 0; bx < gx; ++bx)
                        for (int lp = 0; lp < P; ++lp) {
                            int i, k;
                            if (!dense_diag_pair(f, (long long)bx * P + lp, n, &i, &k)) continue;
                            const int t = la[i], s = la[k];
                            ++pairs[{t < s ? t : s, t < s ? s : t}];
                            write(t, s);
                            write(s, t);  // same launch: the reverse orientation
                        }
            } else {
                for (int t : la)
                    for (int s : lb) {
                        ++pairs[{t < s ? t : s, t < s ? s : t}];
                        write(t, s);  // the reverse goes to the stash and a second launch
                    }
            }
            for (const auto &w : writers)
                if (w.second != 1) {
                    std::printf("FAIL %s entry (%d, %d) written %d times in colour pair (%d, %d)\n", name,
                                w.first.first, w.first.second, w.second, ca, cb);
                    return 1;
                }
        }
    if ((long long)pairs.size() != (long long)nt * (nt - 1) / 2) {
        std::printf("FAIL %s %zu unordered pairs visited, %lld expected\n", name, pairs.size(),
                    (long long)nt * (nt - 1) / 2);
        return 1;
    }
    for (const auto &p : pairs)
        if (p.second != 1) {
            std::printf("FAIL %s pair visited twice\n", name);
            return 1;
        }
    return 0;
}

int main() {
    long long cases = 0;
    for (int n = 2; n <= 300; ++n)
        for (int P : {1, 7, 16}) {
            if (check_fold(n, P)) return 1;
            ++cases;
        }
    for (int n : {511, 512, 1000, 1333}) {
        if (check_fold(n, 16)) return 1;
        ++cases;
    }
    const Mesh meshes[] = {torus(5, 7), torus(12, 9), random_soup(12, 60, 1), random_soup(40, 150, 2), fan(9),
                           fan(3)};
    const char *names[] = {"torus 5x7", "torus 12x9", "soup 12/60", "soup 40/150", "fan 9", "fan 3"};
    for (int i = 0; i < 6; ++i) {
        if (check_mesh(meshes[i], names[i])) return 1;
        ++cases;
    }
    std::printf("ok %lld\n", cases);
    return 0;
}
