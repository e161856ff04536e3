// Host-side FP64 construction of the solver's level data (runs once per
// problem, before any solve).  See setup.h.
#include "setup.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>
#include <sstream>
#include <thread>

namespace glls {

namespace {

// Runs fn(i) for i in [0, count) on up to `threads` host threads.
void parallel_for(long long count, int threads, const std::function<void(long long)>& fn) {
    const int nt = (int)std::max(1LL, std::min<long long>(count, threads));
    if (nt <= 1) {
        for (long long i = 0; i < count; ++i) fn(i);
        return;
    }
    std::atomic<long long> next(0);
    auto work = [&]() {
        for (long long i = next.fetch_add(1); i < count; i = next.fetch_add(1)) fn(i);
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(work);
    work();
    for (auto& t : th) t.join();
}

int host_threads() { return (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency())); }


// Legendre L_p and L_p' at x by the recurrences
//   (n+1) L_{n+1} = (2n+1) x L_n - n L_{n-1},   L_{n+1}' = L_{n-1}' + (2n+1) L_n.
void legendre(int p, double x, double* L, double* dL) {
    double l0 = 1.0, l1 = x, d0 = 0.0, d1 = 1.0;
    if (p == 0) { *L = 1.0; *dL = 0.0; return; }
    for (int n = 1; n < p; ++n) {
        double l2 = ((2 * n + 1) * x * l1 - n * l0) / (n + 1);
        double d2 = d0 + (2 * n + 1) * l1;
        l0 = l1; l1 = l2; d0 = d1; d1 = d2;
    }
    *L = l1;
    *dL = d1;
}

int comp_index(int dim, int a, int b) {
    if (a > b) std::swap(a, b);
    if (dim == 2) return a == 0 ? b : 2;              // 00->0, 01->1, 11->2
    static const int t[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    return t[a][b];
}

// dense (rows x cols) row-major -> banded rows
Band1D to_band(const std::vector<double>& M, int rows, int cols) {
    Band1D b;
    b.rows = rows;
    b.cols = cols;
    b.start.assign(rows, 0);
    int width = 1;
    std::vector<int> lo(rows), hi(rows);
    for (int r = 0; r < rows; ++r) {
        int l = cols, h = -1;
        for (int c = 0; c < cols; ++c)
            if (M[(size_t)r * cols + c] != 0.0) { l = std::min(l, c); h = std::max(h, c); }
        if (h < 0) { l = 0; h = 0; }
        lo[r] = l; hi[r] = h;
        width = std::max(width, h - l + 1);
    }
    b.width = width;
    b.coef.assign((size_t)rows * width, 0.0);
    for (int r = 0; r < rows; ++r) {
        int s = std::min(lo[r], cols - width);
        if (s < 0) s = 0;
        b.start[r] = s;
        for (int k = 0; k < width && s + k < cols; ++k) b.coef[(size_t)r * width + k] = M[(size_t)r * cols + s + k];
    }
    return b;
}

// 1-D global interpolation (ne*p_to + 1) x (ne*p_from + 1): a continuous
// piecewise degree-p_from field sampled at the GLL(p_to) nodes of each element.
std::vector<double> global_interp(int ne, int p_from, int p_to) {
    std::vector<double> J = interpolation(p_from, p_to);
    int rows = ne * p_to + 1, cols = ne * p_from + 1;
    std::vector<double> M((size_t)rows * cols, 0.0);
    for (int e = 0; e < ne; ++e)
        for (int i = 0; i <= p_to; ++i)
            for (int k = 0; k <= p_from; ++k)
                M[(size_t)(e * p_to + i) * cols + e * p_from + k] = J[i * (p_from + 1) + k];
    return M;
}

struct Geo {
    int dim, p, n1, nloc;
    const LevelHost* lv;
    long long gnode(const int ec[3], const int lc[3]) const {
        long long I = (long long)ec[0] * p + lc[0];
        long long J = (long long)ec[1] * p + lc[1];
        long long K = dim == 3 ? (long long)ec[2] * p + lc[2] : 0;
        return (K * lv->n[1] + J) * lv->n[0] + I;
    }
};

void element_coords(const LevelHost& lv, long long e, int ec[3]) {
    ec[0] = (int)(e % lv.ne[0]);
    ec[1] = (int)((e / lv.ne[0]) % lv.ne[1]);
    ec[2] = (int)(e / ((long long)lv.ne[0] * lv.ne[1]));
}

void local_coords(int q, int n1, int dim, int lc[3]) {
    lc[0] = q % n1;
    lc[1] = (q / n1) % n1;
    lc[2] = dim == 3 ? q / (n1 * n1) : 0;
}

int local_index(const int lc[3], int n1) { return (lc[2] * n1 + lc[1]) * n1 + lc[0]; }

// Runs fn(e) for every element e, the elements of one parity colour (the
// parities of its element coordinates) at a time, in parallel: two elements
// of one colour share no node, so per-node accumulation needs no locking.
void for_elements_colored(const LevelHost& lv, const std::function<void(long long)>& fn) {
    const int d = lv.dim;
    for (int c = 0; c < (1 << d); ++c) {
        const long long h[3] = {(lv.ne[0] - (c & 1) + 1) / 2, (lv.ne[1] - ((c >> 1) & 1) + 1) / 2,
                                d == 3 ? (lv.ne[2] - ((c >> 2) & 1) + 1) / 2 : 1};
        const long long cnt = h[0] * h[1] * h[2];
        parallel_for(cnt, host_threads(), [&](long long i) {
            const long long ex = 2 * (i % h[0]) + (c & 1);
            const long long ey = 2 * ((i / h[0]) % h[1]) + ((c >> 1) & 1);
            const long long ez = d == 3 ? 2 * (i / (h[0] * h[1])) + ((c >> 2) & 1) : 0;
            fn((ez * lv.ne[1] + ey) * lv.ne[0] + ex);
        });
    }
}

std::string geometry(LevelHost& lv) {
    const int d = lv.dim, p = lv.p, n1 = p + 1, nloc = lv.nloc;
    std::vector<double> w1;
    gll_nodes(p, &w1);
    lv.D = derivative_matrix(p);
    lv.G.assign((size_t)lv.ncomp * lv.E * nloc, 0.0);
    lv.mass.assign(lv.N, 0.0);
    Geo geo{d, p, n1, nloc, &lv};
    std::mutex err_m;
    std::string err;
    for_elements_colored(lv, [&](long long e) {
        std::vector<double> X((size_t)d * nloc);
        int ec[3];
        element_coords(lv, e, ec);
        for (int q = 0; q < nloc; ++q) {
            int lc[3];
            local_coords(q, n1, d, lc);
            long long g = geo.gnode(ec, lc);
            for (int b = 0; b < d; ++b) X[(size_t)b * nloc + q] = lv.coords[(size_t)b * lv.N + g];
        }
        for (int q = 0; q < nloc; ++q) {
            int lc[3];
            local_coords(q, n1, d, lc);
            double Jm[3][3] = {{0}};   // Jm[b][a] = dx_b / dr_a
            for (int a = 0; a < d; ++a) {
                for (int m = 0; m < n1; ++m) {
                    int mc[3] = {lc[0], lc[1], lc[2]};
                    mc[a] = m;
                    int qm = local_index(mc, n1);
                    double dm = lv.D[lc[a] * n1 + m];
                    for (int b = 0; b < d; ++b) Jm[b][a] += dm * X[(size_t)b * nloc + qm];
                }
            }
            double det, inv[3][3];   // inv[a][c] = dr_a / dx_c
            if (d == 2) {
                det = Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0];
                inv[0][0] = Jm[1][1] / det;  inv[0][1] = -Jm[0][1] / det;
                inv[1][0] = -Jm[1][0] / det; inv[1][1] = Jm[0][0] / det;
            } else {
                double c00 = Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1];
                double c01 = Jm[1][2] * Jm[2][0] - Jm[1][0] * Jm[2][2];
                double c02 = Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0];
                det = Jm[0][0] * c00 + Jm[0][1] * c01 + Jm[0][2] * c02;
                // inverse = adjugate / det; adj[a][c] = cofactor[c][a]
                inv[0][0] = c00 / det;
                inv[1][0] = c01 / det;
                inv[2][0] = c02 / det;
                inv[0][1] = (Jm[0][2] * Jm[2][1] - Jm[0][1] * Jm[2][2]) / det;
                inv[1][1] = (Jm[0][0] * Jm[2][2] - Jm[0][2] * Jm[2][0]) / det;
                inv[2][1] = (Jm[0][1] * Jm[2][0] - Jm[0][0] * Jm[2][1]) / det;
                inv[0][2] = (Jm[0][1] * Jm[1][2] - Jm[0][2] * Jm[1][1]) / det;
                inv[1][2] = (Jm[0][2] * Jm[1][0] - Jm[0][0] * Jm[1][2]) / det;
                inv[2][2] = (Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0]) / det;
            }
            if (!(det > 0.0)) {
                std::ostringstream os;
                os << "non-positive Jacobian " << det << " in element " << e << " (order " << p << ")";
                std::lock_guard<std::mutex> lock(err_m);
                if (err.empty()) err = os.str();
                return;
            }
            double w = 1.0;
            for (int a = 0; a < d; ++a) w *= w1[lc[a]];
            for (int a = 0; a < d; ++a)
                for (int b = a; b < d; ++b) {
                    double s = 0.0;
                    for (int c = 0; c < d; ++c) s += inv[a][c] * inv[b][c];
                    lv.G[(size_t)comp_index(d, a, b) * lv.E * nloc + (size_t)e * nloc + q] = w * det * s;
                }
            lv.mass[geo.gnode(ec, lc)] += w * det;
        }
    });
    return err;
}

inline double Gc(const LevelHost& lv, int a, int b, long long e, int q) {
    return lv.G[(size_t)comp_index(lv.dim, a, b) * lv.E * lv.nloc + (size_t)e * lv.nloc + q];
}

// Band-1 entries of the assembled GLL stiffness (eq. discreteBilinear with
// the nodal basis): diagonal and couplings to the next node along each axis.
void gll_band(LevelHost& lv) {
    const int d = lv.dim, p = lv.p, n1 = p + 1, nloc = lv.nloc;
    const std::vector<double>& D = lv.D;
    lv.diag.assign(lv.N, 0.0);
    for (int s = 0; s < 3; ++s) lv.off[s].assign(lv.N, 0.0);
    Geo geo{d, p, n1, nloc, &lv};
    for_elements_colored(lv, [&](long long e) {
        int ec[3];
        element_coords(lv, e, ec);
        for (int q = 0; q < nloc; ++q) {
            int lc[3];
            local_coords(q, n1, d, lc);
            double v = 0.0;
            for (int a = 0; a < d; ++a) {
                for (int k = 0; k < n1; ++k) {       // sum over quadrature points along a
                    int qc[3] = {lc[0], lc[1], lc[2]};
                    qc[a] = k;
                    double Dk = D[k * n1 + lc[a]];
                    v += Gc(lv, a, a, e, local_index(qc, n1)) * Dk * Dk;
                }
                for (int b = 0; b < d; ++b)
                    if (b != a) v += Gc(lv, a, b, e, q) * D[lc[a] * n1 + lc[a]] * D[lc[b] * n1 + lc[b]];
            }
            long long g = geo.gnode(ec, lc);
            lv.diag[g] += v;
            for (int s = 0; s < d; ++s) {
                if (lc[s] == p) continue;
                const int ms = lc[s];
                double o = 0.0;
                for (int k = 0; k < n1; ++k) {
                    int qc[3] = {lc[0], lc[1], lc[2]};
                    qc[s] = k;
                    o += Gc(lv, s, s, e, local_index(qc, n1)) * D[k * n1 + ms] * D[k * n1 + ms + 1];
                }
                int up[3] = {lc[0], lc[1], lc[2]};
                up[s] = ms + 1;
                int qup = local_index(up, n1);
                for (int b = 0; b < d; ++b) {
                    if (b == s) continue;
                    double Dbb = D[lc[b] * n1 + lc[b]];
                    o += Gc(lv, s, b, e, qup) * D[(ms + 1) * n1 + ms] * Dbb;
                    o += Gc(lv, b, s, e, q) * Dbb * D[ms * n1 + ms + 1];
                }
                lv.off[s][g] += o;
            }
        }
    });
}

// Def. 3.2's line system of an interior grid line is R A_p P: every coupling
// of A_p between two nodes of the line.  Two nodes of a line couple only
// through elements holding both, i.e. within one element segment of p
// intervals, so the system is the sum over the segments of (p+1) x (p+1)
// blocks that overlap at the element-boundary vertices.  Ordering the
// element-interior nodes of every segment first, one step of Algorithm 1 with
// S = the block diagonal of the segment interiors (Thm. 3.8: exact when S
// inverts those blocks exactly) leaves the Schur complement on the vertices
// (Prop. 3.7), a tridiagonal system solved by cyclic reduction (Cor. 3.9).
// This stores, per segment, K_I^-1 and the vertex interpolation weights
// w = K_I^-1 K_{I,v} (the columns of -P restricted to the segment), and per
// line the vertex Schur complement.
//
// Entries of an element's stiffness between nodes m, m' of one local line
// along s (eq. discreteBilinear with the nodal basis, m and m' differing only
// in the s index i, i'):
//   sum_q G_ss(q) D[q,i] D[q,i']                         (q along the line)
// + sum_{b != s} ( D[i',i] G_sb(m') + G_bs(m) D[i,i'] ) D[m_b,m_b]
// for i != i'; the diagonal is the element's full diagonal entry.

struct SegBuilder {
    const LevelHost& lv;
    int s, o1, o2, p, n1, E;
    // element contribution on the local line of element ec through local
    // other indices lc (lc[s] ignored), added into M ((p+1) x (p+1))
    void add_element(const int ec[3], const int lc_in[3], double* M) const {
        const int d = lv.dim;
        const std::vector<double>& D = lv.D;
        long long e = ((long long)ec[2] * lv.ne[1] + ec[1]) * lv.ne[0] + ec[0];
        int lc[3] = {lc_in[0], lc_in[1], lc_in[2]};
        std::vector<int> qv(n1);   // local node index of the line nodes
        for (int i = 0; i < n1; ++i) {
            lc[s] = i;
            qv[i] = local_index(lc, n1);
        }
        for (int i = 0; i < n1; ++i) {
            // full diagonal entry of the element at line node i
            lc[s] = i;
            double v = 0.0;
            for (int a = 0; a < d; ++a) {
                for (int k = 0; k < n1; ++k) {
                    int qc[3] = {lc[0], lc[1], lc[2]};
                    qc[a] = k;
                    double Dk = D[k * n1 + lc[a]];
                    v += Gc(lv, a, a, e, local_index(qc, n1)) * Dk * Dk;
                }
                for (int b = 0; b < d; ++b)
                    if (b != a) v += Gc(lv, a, b, e, qv[i]) * D[lc[a] * n1 + lc[a]] * D[lc[b] * n1 + lc[b]];
            }
            M[i * n1 + i] += v;
            for (int i2 = i + 1; i2 < n1; ++i2) {
                double o = 0.0;
                for (int q = 0; q < n1; ++q) o += Gc(lv, s, s, e, qv[q]) * D[q * n1 + i] * D[q * n1 + i2];
                for (int b = 0; b < d; ++b) {
                    if (b == s) continue;
                    const double Dbb = D[lc_in[b] * n1 + lc_in[b]];
                    o += (D[i2 * n1 + i] * Gc(lv, s, b, e, qv[i2]) + Gc(lv, b, s, e, qv[i]) * D[i * n1 + i2]) * Dbb;
                }
                M[i * n1 + i2] += o;
                M[i2 * n1 + i] += o;
            }
        }
    }
    // summed segment block of line (c1, c2) (global other indices) and segment seg
    void segment(int c1, int c2, int seg, double* M) const {
        std::fill(M, M + n1 * n1, 0.0);
        const int d = lv.dim;
        int e1[2], l1[2], n1c = 0, e2[2] = {0, 0}, l2[2] = {0, 0}, n2c = 1;
        // elements along o1 (and o2) containing the global index c
        auto holders = [&](int c, int a, int* ee, int* ll) {
            int cnt = 0;
            if (c % p == 0) {
                if (c / p - 1 >= 0) { ee[cnt] = c / p - 1; ll[cnt] = p; ++cnt; }
                if (c / p < lv.ne[a]) { ee[cnt] = c / p; ll[cnt] = 0; ++cnt; }
            } else {
                ee[cnt] = c / p; ll[cnt] = c % p; ++cnt;
            }
            return cnt;
        };
        n1c = holders(c1, o1, e1, l1);
        if (d == 3) n2c = holders(c2, o2, e2, l2);
        for (int a = 0; a < n1c; ++a)
            for (int b = 0; b < n2c; ++b) {
                int ec[3] = {0, 0, 0}, lc[3] = {0, 0, 0};
                ec[s] = seg;
                ec[o1] = e1[a];
                lc[o1] = l1[a];
                if (d == 3) { ec[o2] = e2[b]; lc[o2] = l2[b]; }
                add_element(ec, lc, M);
            }
    }
};

// Cholesky inverse of the SPD matrix K (m x m, row-major, overwritten by the
// inverse).  Returns false on a non-positive pivot.
bool spd_inverse_small(double* K, int m) {
    std::vector<double> L((size_t)m * m, 0.0), X((size_t)m * m, 0.0);
    for (int j = 0; j < m; ++j) {
        double s = K[j * m + j];
        for (int k = 0; k < j; ++k) s -= L[j * m + k] * L[j * m + k];
        if (!(s > 0.0)) return false;
        const double ljj = std::sqrt(s);
        L[j * m + j] = ljj;
        for (int i = j + 1; i < m; ++i) {
            double t = K[i * m + j];
            for (int k = 0; k < j; ++k) t -= L[i * m + k] * L[j * m + k];
            L[i * m + j] = t / ljj;
        }
    }
    for (int c = 0; c < m; ++c) {
        std::vector<double> y(m, 0.0);
        for (int i = 0; i < m; ++i) {
            double t = i == c ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) t -= L[i * m + k] * y[k];
            y[i] = t / L[i * m + i];
        }
        for (int i = m - 1; i >= 0; --i) {
            double t = y[i];
            for (int k = i + 1; k < m; ++k) t -= L[k * m + i] * X[k * m + c];
            X[i * m + c] = t / L[i * m + i];
        }
    }
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) K[i * m + j] = 0.5 * (X[i * m + j] + X[j * m + i]);
    return true;
}

std::string line_blocks(LevelHost& lv) {
    const int d = lv.dim, p = lv.p, n1 = p + 1, mi = p - 1;
    lv.lblock = 0;
    if (p < 2) return "";
    const int npk = mi * (mi + 1) / 2, ncoef = npk + 2 * mi;
    for (int s = 0; s < d; ++s) {
        int o1, o2;
        if (s == 0) { o1 = 1; o2 = 2; } else if (s == 1) { o1 = 0; o2 = 2; } else { o1 = 0; o2 = 1; }
        const int m1 = lv.n[o1] - 2, m2 = d == 3 ? lv.n[o2] - 2 : 1;
        const int E = lv.ne[s];
        const long long nlines = (long long)std::max(m1, 0) * std::max(m2, 0);
        const long long ntask = nlines * E;
        lv.blk[s].assign((size_t)ncoef * ntask, 0.0);
        lv.vband[s].assign((size_t)nlines * std::max(E - 1, 0) * 2, 0.0);
        SegBuilder sb{lv, s, o1, o2, p, n1, E};
        std::atomic<long long> next(0);
        std::atomic<bool> bad(false);
        auto work = [&]() {
            std::vector<double> M((size_t)E * n1 * n1), K((size_t)mi * mi);
            std::vector<double> wl((size_t)E * mi), wr((size_t)E * mi);
            for (;;) {
                const long long li = next.fetch_add(1);
                if (li >= nlines || bad.load()) break;
                const int c1 = (int)(li % m1) + 1, c2 = (int)(li / m1) + 1;
                for (int e = 0; e < E; ++e) sb.segment(c1, c2, e, &M[(size_t)e * n1 * n1]);
                for (int e = 0; e < E; ++e) {
                    const double* Me = &M[(size_t)e * n1 * n1];
                    for (int i = 0; i < mi; ++i)
                        for (int j = 0; j < mi; ++j) K[i * mi + j] = Me[(i + 1) * n1 + j + 1];
                    if (!spd_inverse_small(K.data(), mi)) { bad = true; break; }
                    const long long t = li * E + e;
                    int c = 0;
                    for (int i = 0; i < mi; ++i)
                        for (int j = i; j < mi; ++j) lv.blk[s][(size_t)(c++) * ntask + t] = K[i * mi + j];
                    for (int i = 0; i < mi; ++i) {
                        double a = 0.0, b = 0.0;
                        for (int j = 0; j < mi; ++j) {
                            a += K[i * mi + j] * Me[(j + 1) * n1 + 0];
                            b += K[i * mi + j] * Me[(j + 1) * n1 + p];
                        }
                        if (e == 0) a = 0.0;        // left end of the line: boundary node
                        if (e == E - 1) b = 0.0;    // right end
                        wl[(size_t)e * mi + i] = a;
                        wr[(size_t)e * mi + i] = b;
                        lv.blk[s][(size_t)(npk + i) * ntask + t] = a;
                        lv.blk[s][(size_t)(npk + mi + i) * ntask + t] = b;
                    }
                }
                if (bad.load()) break;
                // vertex Schur complement: v = 1 .. E-1 between segments v-1 and v
                for (int v = 1; v < E; ++v) {
                    const double* Ml = &M[(size_t)(v - 1) * n1 * n1];
                    const double* Mr = &M[(size_t)v * n1 * n1];
                    double dg = Ml[p * n1 + p] + Mr[0];
                    for (int i = 0; i < mi; ++i) {
                        dg -= Ml[p * n1 + i + 1] * wr[(size_t)(v - 1) * mi + i];
                        dg -= Mr[0 * n1 + i + 1] * wl[(size_t)v * mi + i];
                    }
                    double of = 0.0;
                    if (v + 1 < E) {
                        of = Mr[0 * n1 + p];
                        for (int i = 0; i < mi; ++i) of -= Mr[0 * n1 + i + 1] * wr[(size_t)v * mi + i];
                    }
                    lv.vband[s][((size_t)li * (E - 1) + (v - 1)) * 2 + 0] = dg;
                    lv.vband[s][((size_t)li * (E - 1) + (v - 1)) * 2 + 1] = of;
                }
            }
        };
        unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        if (nlines < 64) nt = 1;
        std::vector<std::thread> th;
        for (unsigned k = 1; k < nt; ++k) th.emplace_back(work);
        work();
        for (auto& t : th) t.join();
        if (bad.load()) {
            std::ostringstream os;
            os << "line block of order " << p << " along axis " << s << " is not positive definite";
            return os.str();
        }
    }
    lv.lblock = 1;
    return "";
}

// Band-1 entries of the bilinear (trilinear) FEM matrix on the mesh of GLL
// nodes, each cell a Q1 element on its physical vertices, 2-point Gauss rule.
void fem_band(LevelHost& lv) {
    const int d = lv.dim;
    lv.diag.assign(lv.N, 0.0);
    for (int s = 0; s < 3; ++s) lv.off[s].assign(lv.N, 0.0);
    const int nc = 1 << d;
    const double gp[2] = {-1.0 / std::sqrt(3.0), 1.0 / std::sqrt(3.0)};
    int cn[3] = {lv.n[0] - 1, lv.n[1] - 1, d == 3 ? lv.n[2] - 1 : 1};
    for (int ck = 0; ck < cn[2]; ++ck)
        for (int cj = 0; cj < cn[1]; ++cj)
            for (int ci = 0; ci < cn[0]; ++ci) {
                long long node[8];
                double X[3][8];
                for (int c = 0; c < nc; ++c) {
                    int o0 = c & 1, o1 = (c >> 1) & 1, o2 = (c >> 2) & 1;
                    long long g = ((long long)(ck + o2) * lv.n[1] + (cj + o1)) * lv.n[0] + (ci + o0);
                    node[c] = g;
                    for (int b = 0; b < d; ++b) X[b][c] = lv.coords[(size_t)b * lv.N + g];
                }
                double K[8][8] = {{0}};
                for (int qp = 0; qp < nc; ++qp) {
                    double r[3] = {gp[qp & 1], gp[(qp >> 1) & 1], gp[(qp >> 2) & 1]};
                    double dN[8][3];
                    for (int c = 0; c < nc; ++c) {
                        double sgn[3] = {(c & 1) ? 1.0 : -1.0, ((c >> 1) & 1) ? 1.0 : -1.0, ((c >> 2) & 1) ? 1.0 : -1.0};
                        for (int t = 0; t < d; ++t) {
                            double v = 0.5 * sgn[t];
                            for (int t2 = 0; t2 < d; ++t2)
                                if (t2 != t) v *= 0.5 * (1.0 + sgn[t2] * r[t2]);
                            dN[c][t] = v;
                        }
                    }
                    double Jm[3][3] = {{0}};
                    for (int b = 0; b < d; ++b)
                        for (int t = 0; t < d; ++t)
                            for (int c = 0; c < nc; ++c) Jm[b][t] += X[b][c] * dN[c][t];
                    double det, inv[3][3];
                    if (d == 2) {
                        det = Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0];
                        inv[0][0] = Jm[1][1] / det;  inv[0][1] = -Jm[0][1] / det;
                        inv[1][0] = -Jm[1][0] / det; inv[1][1] = Jm[0][0] / det;
                    } else {
                        double c00 = Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1];
                        double c01 = Jm[1][2] * Jm[2][0] - Jm[1][0] * Jm[2][2];
                        double c02 = Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0];
                        det = Jm[0][0] * c00 + Jm[0][1] * c01 + Jm[0][2] * c02;
                        inv[0][0] = c00 / det; inv[1][0] = c01 / det; inv[2][0] = c02 / det;
                        inv[0][1] = (Jm[0][2] * Jm[2][1] - Jm[0][1] * Jm[2][2]) / det;
                        inv[1][1] = (Jm[0][0] * Jm[2][2] - Jm[0][2] * Jm[2][0]) / det;
                        inv[2][1] = (Jm[0][1] * Jm[2][0] - Jm[0][0] * Jm[2][1]) / det;
                        inv[0][2] = (Jm[0][1] * Jm[1][2] - Jm[0][2] * Jm[1][1]) / det;
                        inv[1][2] = (Jm[0][2] * Jm[1][0] - Jm[0][0] * Jm[1][2]) / det;
                        inv[2][2] = (Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0]) / det;
                    }
                    double gx[8][3];
                    for (int c = 0; c < nc; ++c)
                        for (int b = 0; b < d; ++b) {
                            double v = 0.0;
                            for (int t = 0; t < d; ++t) v += dN[c][t] * inv[t][b];
                            gx[c][b] = v;
                        }
                    for (int c = 0; c < nc; ++c)
                        for (int c2 = 0; c2 < nc; ++c2) {
                            double v = 0.0;
                            for (int b = 0; b < d; ++b) v += gx[c][b] * gx[c2][b];
                            K[c][c2] += v * std::fabs(det);
                        }
                }
                for (int c = 0; c < nc; ++c) {
                    lv.diag[node[c]] += K[c][c];
                    for (int s = 0; s < d; ++s)
                        if (!((c >> s) & 1)) lv.off[s][node[c]] += K[c][c | (1 << s)];
                }
            }
}

}  // namespace

std::vector<double> gll_nodes(int p, std::vector<double>* weights) {
    std::vector<double> xi(p + 1);
    xi[0] = -1.0;
    xi[p] = 1.0;
    const double pi = 3.14159265358979323846;
    for (int n = 1; n < p; ++n) {
        double x = -std::cos(pi * n / p);
        for (int it = 0; it < 100; ++it) {
            double L, dL;
            legendre(p, x, &L, &dL);
            // Newton on L_p'(x); L_p'' from Legendre's equation
            double d2L = (2.0 * x * dL - p * (p + 1.0) * L) / (1.0 - x * x);
            double step = dL / d2L;
            x -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        xi[n] = x;
    }
    if (weights) {
        weights->assign(p + 1, 0.0);
        for (int n = 0; n <= p; ++n) {
            double L, dL;
            legendre(p, xi[n], &L, &dL);
            (*weights)[n] = 2.0 / (p * (p + 1.0) * L * L);
        }
    }
    return xi;
}

// D[i][j] = pi_j'(xi_i) from the closed form in Legendre values:
// L_p(xi_i) / (L_p(xi_j) (xi_i - xi_j)) off the diagonal, -+p(p+1)/4 at the ends.
std::vector<double> derivative_matrix(int p) {
    std::vector<double> xi = gll_nodes(p, nullptr);
    std::vector<double> L(p + 1);
    for (int i = 0; i <= p; ++i) {
        double dl;
        legendre(p, xi[i], &L[i], &dl);
    }
    std::vector<double> D((p + 1) * (p + 1), 0.0);
    for (int i = 0; i <= p; ++i)
        for (int j = 0; j <= p; ++j)
            if (i != j) D[i * (p + 1) + j] = L[i] / (L[j] * (xi[i] - xi[j]));
    D[0] = -p * (p + 1) / 4.0;
    D[p * (p + 1) + p] = p * (p + 1) / 4.0;
    return D;
}

std::vector<double> interpolation(int p_from, int p_to) {
    std::vector<double> xf = gll_nodes(p_from, nullptr), xt = gll_nodes(p_to, nullptr);
    std::vector<double> J((p_to + 1) * (p_from + 1));
    for (int i = 0; i <= p_to; ++i)
        for (int k = 0; k <= p_from; ++k) {
            double v = 1.0;
            for (int m = 0; m <= p_from; ++m)
                if (m != k) v *= (xt[i] - xf[m]) / (xf[k] - xf[m]);
            J[i * (p_from + 1) + k] = v;
        }
    return J;
}

std::vector<int> order_chain(int p_fine, bool multi) {
    int p0 = multi ? 1 : 2;
    std::vector<int> c{p_fine};
    while (c.back() > p0) c.push_back(std::max(p0, c.back() / 2));
    return c;
}

std::string build_levels(int dim, const int nelem[3], int p_fine, const double* coords,
                         int smoother, int restriction, std::vector<LevelHost>& levels, double* phase_ms) {
    double local_ms[4] = {0, 0, 0, 0};
    if (!phase_ms) phase_ms = local_ms;
    auto clock_ms = [] {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
    };
    double tp = clock_ms();
    auto lap = [&](int k) {
        const double t = clock_ms();
        phase_ms[k] += t - tp;
        tp = t;
    };
    // p = 1 has interior unknowns only with at least two elements along every axis
    bool multi = nelem[0] > 1 && nelem[1] > 1 && (dim == 2 || nelem[2] > 1);
    std::vector<int> chain = order_chain(p_fine, multi);
    levels.assign(chain.size(), LevelHost());
    // fill from fine (back) to coarse (front)
    for (size_t c = 0; c < chain.size(); ++c) {
        LevelHost& lv = levels[chain.size() - 1 - c];
        lv.dim = dim;
        lv.p = chain[c];
        lv.N = 1;
        lv.E = 1;
        for (int a = 0; a < 3; ++a) {
            lv.ne[a] = a < dim ? nelem[a] : 1;
            lv.n[a] = a < dim ? nelem[a] * lv.p + 1 : 1;
            lv.N *= lv.n[a];
            lv.E *= lv.ne[a];
        }
        lv.nloc = 1;
        for (int a = 0; a < dim; ++a) lv.nloc *= lv.p + 1;
        lv.ncomp = dim == 2 ? 3 : 6;
        lv.coords.assign((size_t)dim * lv.N, 0.0);
        if (c == 0) {
            std::memcpy(lv.coords.data(), coords, sizeof(double) * dim * lv.N);
        } else {
            // coarse nodes: the finer element's coordinate polynomial at coarse
            // GLL points, i.e. the 1-D interpolation J applied along each axis
            // of the element's fine nodal coordinates (sum factorisation)
            const LevelHost& f = levels[chain.size() - c];
            const int pf = f.p, pc = lv.p, n1f = pf + 1, n1c = pc + 1;
            const std::vector<double> J = interpolation(pf, pc);   // [(pc+1) x (pf+1)]
            const int nzf = dim == 3 ? n1f : 1, nzc = dim == 3 ? n1c : 1;
            std::vector<double> a((size_t)nzf * n1f * n1f), b((size_t)nzf * n1f * n1c), cc((size_t)nzf * n1c * n1c),
                out((size_t)nzc * n1c * n1c);
            for (long long e = 0; e < lv.E; ++e) {
                int ec[3];
                element_coords(lv, e, ec);
                for (int bdim = 0; bdim < dim; ++bdim) {
                    for (int k = 0; k < nzf; ++k)
                        for (int j = 0; j < n1f; ++j)
                            for (int i = 0; i < n1f; ++i) {
                                const long long gf = ((long long)(dim == 3 ? ec[2] * pf + k : 0) * f.n[1] + ec[1] * pf + j) *
                                                         f.n[0] + ec[0] * pf + i;
                                a[((size_t)k * n1f + j) * n1f + i] = f.coords[(size_t)bdim * f.N + gf];
                            }
                    // along x, then y, then z
                    for (int k = 0; k < nzf; ++k)
                        for (int j = 0; j < n1f; ++j)
                            for (int i = 0; i < n1c; ++i) {
                                double v = 0.0;
                                for (int q = 0; q < n1f; ++q) v += J[i * n1f + q] * a[((size_t)k * n1f + j) * n1f + q];
                                b[((size_t)k * n1f + j) * n1c + i] = v;
                            }
                    for (int k = 0; k < nzf; ++k)
                        for (int j = 0; j < n1c; ++j)
                            for (int i = 0; i < n1c; ++i) {
                                double v = 0.0;
                                for (int q = 0; q < n1f; ++q) v += J[j * n1f + q] * b[((size_t)k * n1f + q) * n1c + i];
                                cc[((size_t)k * n1c + j) * n1c + i] = v;
                            }
                    for (int k = 0; k < nzc; ++k)
                        for (int j = 0; j < n1c; ++j)
                            for (int i = 0; i < n1c; ++i) {
                                double v = 0.0;
                                if (dim == 3) {
                                    for (int q = 0; q < n1f; ++q) v += J[k * n1f + q] * cc[((size_t)q * n1c + j) * n1c + i];
                                } else {
                                    v = cc[(size_t)j * n1c + i];
                                }
                                const long long gc = ((long long)(dim == 3 ? ec[2] * pc + k : 0) * lv.n[1] + ec[1] * pc + j) *
                                                         lv.n[0] + ec[0] * pc + i;
                                lv.coords[(size_t)bdim * lv.N + gc] = v;
                            }
                }
            }
        }
        lap(0);
        std::string err = geometry(lv);
        lap(1);
        if (!err.empty()) return err;
        if (smoother == 1) {
            fem_band(lv);
        } else {
            gll_band(lv);
            if (smoother == 0) {
                err = line_blocks(lv);
                if (!err.empty()) return err;
            }
        }
        lap(2);
    }
    // transfers between consecutive levels
    for (size_t l = 1; l < levels.size(); ++l) {
        LevelHost& f = levels[l];
        const LevelHost& c = levels[l - 1];
        for (int a = 0; a < dim; ++a) {
            std::vector<double> P = global_interp(f.ne[a], c.p, f.p);     // n_f x n_c
            int nf = f.n[a], ncn = c.n[a];
            f.P[a] = to_band(P, nf, ncn);
            std::vector<double> R((size_t)ncn * nf);
            if (restriction == 0) {
                for (int i = 0; i < nf; ++i)
                    for (int k = 0; k < ncn; ++k) R[(size_t)k * nf + i] = P[(size_t)i * ncn + k];
            } else {
                R = global_interp(f.ne[a], f.p, c.p);                     // n_c x n_f
            }
            f.R[a] = to_band(R, ncn, nf);
        }
    }
    lap(3);
    return "";
}

// Inverse of an SPD matrix with half bandwidth bw (dense n x n row-major):
// banded Cholesky A = L L^T, then L L^T x = e_c for every column c (columns
// split over `threads` host threads).  The back substitution reads a
// transposed copy of the band, and the inverse, being symmetric, is written
// by rows.
std::string spd_band_inverse(const std::vector<double>& A, long long n, long long bw, std::vector<double>& inv,
                             int threads = 1) {
    // banded Cholesky A = L L^T, L stored dense (lower band used)
    std::vector<double> L((size_t)n * n, 0.0);
    for (long long j = 0; j < n; ++j) {
        long long k0 = std::max(0LL, j - bw);
        double s = A[(size_t)j * n + j];
        for (long long k = k0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(s > 0.0)) return "coarsest-level matrix is not positive definite";
        double ljj = std::sqrt(s);
        L[(size_t)j * n + j] = ljj;
        for (long long i = j + 1; i <= std::min(n - 1, j + bw); ++i) {
            double t = A[(size_t)i * n + j];
            long long kk = std::max(k0, i - bw);
            for (long long k = kk; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = t / ljj;
        }
    }
    // U[i][k - i] = L[k][i] for i <= k <= i + bw
    const long long w = bw + 1;
    std::vector<double> U((size_t)n * w, 0.0);
    for (long long i = 0; i < n; ++i)
        for (long long k = i; k <= std::min(n - 1, i + bw); ++k) U[(size_t)i * w + (k - i)] = L[(size_t)k * n + i];
    inv.assign((size_t)n * n, 0.0);
    parallel_for(n, threads, [&](long long c) {
        std::vector<double> y(n, 0.0);
        // forward L y = e_c
        for (long long i = c; i < n; ++i) {
            double t = (i == c) ? 1.0 : 0.0;
            for (long long k = std::max(c, i - bw); k < i; ++k) t -= L[(size_t)i * n + k] * y[k];
            y[i] = t / L[(size_t)i * n + i];
        }
        // backward L^T x = y
        for (long long i = n - 1; i >= 0; --i) {
            double t = y[i];
            const long long kmax = std::min(n - 1, i + bw);
            for (long long k = i + 1; k <= kmax; ++k) t -= U[(size_t)i * w + (k - i)] * y[k];
            y[i] = t / U[(size_t)i * w];
        }
        // A^-1 is symmetric: column c is row c
        std::copy(y.begin(), y.end(), inv.begin() + (size_t)c * n);
    });
    return "";
}

namespace {

using Mat = std::vector<double>;

// C = beta C + alpha op(A) op(B), row-major with leading dimensions: op(A)
// is M x K (A, or A^T stored K x M), op(B) is K x N.  Panels of op(A) (kMR
// rows) and op(B) (kNR columns) are packed per kKC-deep slice so that the
// kMR x kNR register tile of the inner loop streams both contiguously; row
// blocks of kMC rows are split over `threads` host threads.
constexpr int kMR = 4, kNR = 8, kKC = 256, kMC = 64;

void gemm(int M, int N, int K, double alpha, const double* A, int lda, bool transA, const double* B, int ldb,
          bool transB, double beta, double* C, int ldc, int threads = 1) {
    const int nrb = (N + kNR - 1) / kNR;
    std::vector<double> Bp((size_t)nrb * kKC * kNR);
    if (K == 0) {
        for (int i = 0; i < M; ++i)
            for (int j = 0; j < N; ++j) C[(size_t)i * ldc + j] = beta == 0.0 ? 0.0 : beta * C[(size_t)i * ldc + j];
        return;
    }
    for (int k0 = 0; k0 < K; k0 += kKC) {
        const int kc = std::min(kKC, K - k0);
        // pack op(B)[k0 : k0 + kc, :] as nrb panels of [kc][kNR], zero-padded
        for (int jb = 0; jb < nrb; ++jb) {
            double* dst = &Bp[(size_t)jb * kKC * kNR];
            const int j0 = jb * kNR, nj = std::min(kNR, N - j0);
            for (int k = 0; k < kc; ++k)
                for (int j = 0; j < kNR; ++j)
                    dst[k * kNR + j] = j >= nj ? 0.0
                                       : transB ? B[(size_t)(j0 + j) * ldb + k0 + k]
                                                : B[(size_t)(k0 + k) * ldb + j0 + j];
        }
        const bool first = k0 == 0;
        const int nmc = (M + kMC - 1) / kMC;
        parallel_for(nmc, threads, [&](long long ib) {
            const int i0 = (int)ib * kMC, mc = std::min(kMC, M - i0);
            const int nmr = (mc + kMR - 1) / kMR;
            std::vector<double> Ap((size_t)nmr * kc * kMR);
            // pack op(A)[i0 : i0 + mc, k0 : k0 + kc] as panels of [kc][kMR]
            for (int r = 0; r < nmr; ++r)
                for (int k = 0; k < kc; ++k)
                    for (int i = 0; i < kMR; ++i) {
                        const int row = i0 + r * kMR + i;
                        double v = 0.0;
                        if (row < M) v = transA ? A[(size_t)(k0 + k) * lda + row] : A[(size_t)row * lda + k0 + k];
                        Ap[((size_t)r * kc + k) * kMR + i] = v;
                    }
            for (int r = 0; r < nmr; ++r) {
                const int rows = std::min(kMR, mc - r * kMR);
                for (int jb = 0; jb < nrb; ++jb) {
                    const int cols = std::min(kNR, N - jb * kNR);
                    double acc[kMR][kNR] = {};
                    const double* ap = &Ap[(size_t)r * kc * kMR];
                    const double* bp = &Bp[(size_t)jb * kKC * kNR];
                    for (int k = 0; k < kc; ++k) {
#pragma GCC unroll 4
                        for (int i = 0; i < kMR; ++i) {
                            const double ai = ap[k * kMR + i];
#pragma GCC unroll 8
                            for (int j = 0; j < kNR; ++j) acc[i][j] += ai * bp[k * kNR + j];
                        }
                    }
                    for (int i = 0; i < rows; ++i) {
                        double* c = C + (size_t)(i0 + r * kMR + i) * ldc + jb * kNR;
                        for (int j = 0; j < cols; ++j) {
                            const double base = first ? (beta == 0.0 ? 0.0 : beta * c[j]) : c[j];
                            c[j] = base + alpha * acc[i][j];
                        }
                    }
                }
            }
        });
    }
}

// C = beta C + alpha op(A) B for m x m blocks
void gemm(int m, const double* A, bool transA, const double* B, double* C, double alpha, double beta,
          int threads = 1) {
    gemm(m, m, m, alpha, A, m, transA, B, m, false, beta, C, m, threads);
}

// Inverse of the SPD matrix A (n x n, leading dimension lda) into inv (n x
// n, leading dimension ldi) by the 2 x 2 block form with the Schur
// complement S = A22 - A21 A11^-1 A12 (itself SPD):
//   A^-1 = [A11^-1 + X S^-1 X^T, -X S^-1; -S^-1 X^T, S^-1],  X = A11^-1 A12,
// recursively, with the products by gemm; blocks of up to 64 by Cholesky.
bool spd_inverse_blocked(const double* A, int n, int lda, double* inv, int ldi, int threads) {
    if (n <= 64) {
        std::vector<double> K((size_t)n * n);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) K[(size_t)i * n + j] = A[(size_t)i * lda + j];
        if (!spd_inverse_small(K.data(), n)) return false;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) inv[(size_t)i * ldi + j] = K[(size_t)i * n + j];
        return true;
    }
    const int h = (n / 2 + kMR - 1) / kMR * kMR, r = n - h;
    const double* A12 = A + h;
    const double* A21 = A + (size_t)h * lda;
    const double* A22 = A21 + h;
    double* I11 = inv;
    double* I12 = inv + h;
    double* I21 = inv + (size_t)h * ldi;
    double* I22 = I21 + h;
    if (!spd_inverse_blocked(A, h, lda, I11, ldi, threads)) return false;
    std::vector<double> X((size_t)h * r), S((size_t)r * r);
    gemm(h, r, h, 1.0, I11, ldi, false, A12, lda, false, 0.0, X.data(), r, threads);        // X = A11^-1 A12
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < r; ++j) S[(size_t)i * r + j] = A22[(size_t)i * lda + j];
    gemm(r, r, h, -1.0, A21, lda, false, X.data(), r, false, 1.0, S.data(), r, threads);    // S = A22 - A21 X
    if (!spd_inverse_blocked(S.data(), r, r, I22, ldi, threads)) return false;
    gemm(h, r, r, -1.0, X.data(), r, false, I22, ldi, false, 0.0, I12, ldi, threads);      // -X S^-1
    gemm(h, h, r, -1.0, I12, ldi, false, X.data(), r, true, 1.0, I11, ldi, threads);       // + X S^-1 X^T
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < h; ++j) I21[(size_t)i * ldi + j] = I12[(size_t)j * ldi + i];
    return true;
}

// Inverse of an SPD matrix with half bandwidth bw: the banded Cholesky
// solve costs about 2 n^2 bw scalar operations, the blocked dense inverse
// 4/3 n^3 in cache-blocked products (an order of magnitude faster per
// operation), so the dense form is taken unless the band is narrow.
std::string spd_inverse_auto(const std::vector<double>& A, long long n, long long bw, std::vector<double>& inv,
                             int threads) {
    if (n >= 16 * (bw + 1) || n > 46340) return spd_band_inverse(A, n, bw, inv, threads);
    inv.assign((size_t)n * n, 0.0);
    if (!spd_inverse_blocked(A.data(), (int)n, (int)n, inv.data(), (int)n, threads))
        return "coarsest-level matrix is not positive definite";
    for (long long r = 0; r < n; ++r)
        for (long long c = r + 1; c < n; ++c) {
            const double v = 0.5 * (inv[(size_t)r * n + c] + inv[(size_t)c * n + r]);
            inv[(size_t)r * n + c] = inv[(size_t)c * n + r] = v;
        }
    return "";
}

}  // namespace

int max_cr_levels(int nb) {
    int k = 0;
    while ((2 << k) <= nb) ++k;     // at least one block is left after k levels
    return k;
}

// Depth of block CR before the dense solve that minimises a launch-plus-bytes
// model of the GPU solve: each CR level costs a forward and a backward launch
// (about 2 us each) and reads 2 m^2 values per kept block and 3 m^2 per
// eliminated block; the dense solve reads (remaining unknowns)^2 values; FP32
// bytes streamed at 5 TB/s.  0 means the dense inverse of the whole system.
int auto_cr_levels(int nb, int m) {
    const double mm = (double)m * m;
    int best = 0;
    double best_t = 2.0 + 4.0 * ((double)nb * m) * ((double)nb * m) / 5.0e6;
    double level_bytes = 0.0;
    for (int k = 1; k <= max_cr_levels(nb); ++k) {
        const int a = nb >> (k - 1);                 // active blocks at level k - 1
        level_bytes += 4.0 * mm * (2.0 * (a / 2) + 3.0 * ((a + 1) / 2));
        const double nr = (double)(nb >> k) * m;
        const double t = 2.0 * (2 * k + 1) + (level_bytes + 4.0 * nr * nr) / 5.0e6;
        if (t < best_t) {
            best_t = t;
            best = k;
        }
    }
    return best;
}

// Block cyclic reduction of the block-tridiagonal matrix with diagonal blocks
// Ab, sub-diagonal Lb and super-diagonal Ub (Def. 3.5 blocks of size m, nb
// blocks) for k levels (Thm. 3.8 with m > 1, Prop. 3.7, Cor. 3.9), then the
// dense inverse of the remaining coarse system.  At each level the odd blocks
// (1-based) are eliminated: stored A_j^-1, A_j^-1 L_j, A_j^-1 U_j; the even
// blocks are kept: stored L_i A_{i-1}^-1 and U_i A_{i+1}^-1, and their coarse
// blocks follow Prop. 3.7.  The blocks of a level are processed in parallel.
std::string build_block_cr(std::vector<Mat> Ab, std::vector<Mat> Lb, std::vector<Mat> Ub, int m, int k,
                           CoarseHost& out) {
    const int threads = host_threads();
    const size_t mm = (size_t)m * m;
    out.fh.assign(k, Mat());
    out.agk.assign(k, Mat());
    for (int l = 0; l < k; ++l) {
        const int a = (int)Ab.size();
        const int ne = (a + 1) / 2, nk = a / 2;
        out.agk[l].assign(3 * mm * ne, 0.0);
        std::vector<std::string> errs(a);
        const int inner_e = std::max(1, threads / std::max(1, ne));
        parallel_for(ne, threads, [&](long long q) {      // eliminated (1-based odd)
            const int t = (int)(2 * q);
            double* dst = &out.agk[l][3 * mm * q];
            if (!spd_inverse_blocked(Ab[t].data(), m, m, dst, m, inner_e)) {
                errs[t] = "coarsest-level matrix is not positive definite";
                return;
            }
            for (int r = 0; r < m; ++r)          // exactly symmetric
                for (int c = r + 1; c < m; ++c) {
                    const double v = 0.5 * (dst[(size_t)r * m + c] + dst[(size_t)c * m + r]);
                    dst[(size_t)r * m + c] = dst[(size_t)c * m + r] = v;
                }
            gemm(m, dst, false, Lb[t].data(), dst + mm, 1.0, 0.0, inner_e);        // A_j^-1 L_j
            gemm(m, dst, false, Ub[t].data(), dst + 2 * mm, 1.0, 0.0, inner_e);    // A_j^-1 U_j
        });
        for (const auto& e : errs)
            if (!e.empty()) return e;
        // kept blocks.  A_0 is symmetric, so L_i = U_{i-1}^T and
        //   F = L_i A_{i-1}^-1 = (A_{i-1}^-1 U_{i-1})^T,  H = U_i A_{i+1}^-1 = (A_{i+1}^-1 L_{i+1})^T,
        // both already formed for the eliminated neighbours.
        std::vector<Mat> A2(nk), L2(nk), U2(nk);
        out.fh[l].assign(2 * mm * nk, 0.0);
        const int inner_k = std::max(1, threads / std::max(1, nk));
        parallel_for(nk, threads, [&](long long q) {      // kept (1-based even)
            const int t = (int)(2 * q + 1);
            const bool right = t + 1 < a;
            const double* Kl = &out.agk[l][3 * mm * q + 2 * mm];                    // A_{t-1}^-1 U_{t-1}
            const double* Gr = right ? &out.agk[l][3 * mm * (q + 1) + mm] : nullptr; // A_{t+1}^-1 L_{t+1}
            double* dst = &out.fh[l][2 * mm * q];
            for (int r = 0; r < m; ++r)
                for (int c = 0; c < m; ++c) {
                    dst[(size_t)r * m + c] = Kl[(size_t)c * m + r];
                    if (right) dst[mm + (size_t)r * m + c] = Gr[(size_t)c * m + r];
                }
            Mat An = Ab[t];
            gemm(m, Kl, true, Ub[t - 1].data(), An.data(), -1.0, 1.0, inner_k);    // - F U_{t-1}
            L2[q].assign(mm, 0.0);
            gemm(m, Kl, true, Lb[t - 1].data(), L2[q].data(), -1.0, 0.0, inner_k);  // - F L_{t-1}
            U2[q].assign(mm, 0.0);
            if (right) {
                gemm(m, Gr, true, Lb[t + 1].data(), An.data(), -1.0, 1.0, inner_k); // - H L_{t+1}
                gemm(m, Gr, true, Ub[t + 1].data(), U2[q].data(), -1.0, 0.0, inner_k);  // - H U_{t+1}
            }
            A2[q] = std::move(An);
        });
        Ab.swap(A2);
        Lb.swap(L2);
        Ub.swap(U2);
    }
    const int a = (int)Ab.size();
    const long long nr = (long long)a * m;
    out.nr = nr;
    std::vector<double> Ar((size_t)nr * nr, 0.0);
    for (int t = 0; t < a; ++t)
        for (int r = 0; r < m; ++r)
            for (int c = 0; c < m; ++c) {
                const size_t row = (size_t)((long long)t * m + r) * nr;
                Ar[row + (size_t)t * m + c] = Ab[t][(size_t)r * m + c];
                if (t > 0) Ar[row + (size_t)(t - 1) * m + c] = Lb[t][(size_t)r * m + c];
                if (t + 1 < a) Ar[row + (size_t)(t + 1) * m + c] = Ub[t][(size_t)r * m + c];
            }
    return spd_inverse_auto(Ar, nr, std::min<long long>(nr - 1, 2LL * m - 1), out.inv, threads);
}

std::string build_coarse(const LevelHost& lv, int coarse_solver, int cr_levels, CoarseHost& out) {
    const int d = lv.dim, p = lv.p, n1 = p + 1, nloc = lv.nloc;
    std::vector<long long> id(lv.N, -1);
    out.index.clear();
    for (long long g = 0; g < lv.N; ++g) {
        long long I = g % lv.n[0], J = (g / lv.n[0]) % lv.n[1], K = g / ((long long)lv.n[0] * lv.n[1]);
        bool inner = I > 0 && I < lv.n[0] - 1 && J > 0 && J < lv.n[1] - 1 && (d == 2 || (K > 0 && K < lv.n[2] - 1));
        if (inner) { id[g] = (long long)out.index.size(); out.index.push_back(g); }
    }
    const long long n = (long long)out.index.size();
    out.n = n;
    if (n == 0) return "coarsest level has no interior unknowns";
    // blocks: one per interior index of the slowest axis (grid lines in 2-D,
    // planes in 3-D); the lexicographic numbering makes them contiguous, and
    // A_0 couples a block only to itself and its two neighbours
    out.nb = lv.n[d - 1] - 2;
    out.m = (int)(n / out.nb);
    // at p > 1 (a grid with one element along some axis stops at p = 2) a
    // node couples to nodes up to p slowest-axis indices away: the system is
    // not block tridiagonal over those indices, and the dense inverse is used
    const bool block_tridiagonal = p == 1;
    const int nb = block_tridiagonal ? out.nb : 1, m = block_tridiagonal ? out.m : (int)n;
    if (!block_tridiagonal) {
        out.nb = 1;
        out.m = (int)n;
    }
    int k = 0;
    if (!block_tridiagonal) k = 0;
    else if (coarse_solver == 2)
        k = std::min(cr_levels > 0 ? cr_levels : std::max(1, auto_cr_levels(nb, m)), max_cr_levels(nb));
    else if (coarse_solver == 0) k = auto_cr_levels(nb, m);
    // the dense inverse of the whole system is kept to moderate sizes; larger
    // systems take at least one level of block CR
    constexpr long long kMaxDenseUnknowns = 16384;
    if (k == 0 && n > kMaxDenseUnknowns) {
        if (coarse_solver == 1 || !block_tridiagonal)
            return "coarsest level has more than 16384 interior unknowns: use GLLS_COARSE_AUTO or GLLS_COARSE_BLOCK_CR";
        k = std::max(1, std::min(max_cr_levels(nb), auto_cr_levels(nb, m)));
    }
    if (k == 0 && n > kMaxDenseUnknowns) return "coarsest level too large for a dense inverse";
    // block CR stores dense m x m blocks: bound their size and number
    constexpr int kMaxBlock = 2048;
    if (k > 0 && (m > kMaxBlock || (double)nb * m * m * 8.0 * 6.0 > 24e9))
        return "coarsest level too large for block cyclic reduction (blocks of " + std::to_string(m) + " unknowns)";
    out.cr_levels = k;
    // assemble the blocks from the element matrices:
    // A_e[m][m2] = sum_q sum_ab G_ab(q) B_a(q, m) B_b(q, m2)
    const size_t mm = (size_t)m * m;
    // (one block: the whole system, no coupling blocks)
    std::vector<Mat> Ab(nb, Mat(mm, 0.0)), Lb(nb, Mat(nb > 1 ? mm : 0, 0.0)), Ub(nb, Mat(nb > 1 ? mm : 0, 0.0));
    long long bw = 0;
    Geo geo{d, p, n1, nloc, &lv};
    const std::vector<double>& D = lv.D;
    for (long long e = 0; e < lv.E; ++e) {
        int ec[3];
        element_coords(lv, e, ec);
        for (int mq = 0; mq < nloc; ++mq) {
            int mc[3];
            local_coords(mq, n1, d, mc);
            long long gm = id[geo.gnode(ec, mc)];
            if (gm < 0) continue;
            for (int m2 = 0; m2 < nloc; ++m2) {
                int mc2[3];
                local_coords(m2, n1, d, mc2);
                long long gm2 = id[geo.gnode(ec, mc2)];
                if (gm2 < 0) continue;
                double v = 0.0;
                for (int q = 0; q < nloc; ++q) {
                    int qc[3];
                    local_coords(q, n1, d, qc);
                    for (int a = 0; a < d; ++a) {
                        bool oka = true;
                        for (int c = 0; c < d; ++c) if (c != a && qc[c] != mc[c]) oka = false;
                        if (!oka) continue;
                        double Ba = D[qc[a] * n1 + mc[a]];
                        for (int b = 0; b < d; ++b) {
                            bool okb = true;
                            for (int c = 0; c < d; ++c) if (c != b && qc[c] != mc2[c]) okb = false;
                            if (!okb) continue;
                            v += Gc(lv, a, b, e, q) * Ba * D[qc[b] * n1 + mc2[b]];
                        }
                    }
                }
                const long long bi = gm / m, bj = gm2 / m;
                const size_t o = (size_t)(gm % m) * m + (size_t)(gm2 % m);
                if (bj == bi) Ab[bi][o] += v;
                else if (bj == bi - 1) Lb[bi][o] += v;
                else if (bj == bi + 1) Ub[bi][o] += v;
                else return "coarsest-level matrix is not block tridiagonal over the slowest axis";
                bw = std::max(bw, std::llabs(gm - gm2));
            }
        }
    }
    if (k == 0) {       // dense A_0^-1
        std::vector<double> A((size_t)n * n, 0.0);
        for (int t = 0; t < nb; ++t)
            for (int r = 0; r < m; ++r)
                for (int c = 0; c < m; ++c) {
                    const size_t row = (size_t)((long long)t * m + r) * n;
                    A[row + (size_t)t * m + c] = Ab[t][(size_t)r * m + c];
                    if (t > 0) A[row + (size_t)(t - 1) * m + c] = Lb[t][(size_t)r * m + c];
                    if (t + 1 < nb) A[row + (size_t)(t + 1) * m + c] = Ub[t][(size_t)r * m + c];
                }
        out.nr = n;
        return spd_inverse_auto(A, n, bw, out.inv, host_threads());
    }
    return build_block_cr(std::move(Ab), std::move(Lb), std::move(Ub), m, k, out);
}

}  // namespace glls
