// Host-side (FP64) construction of the level data of the GLL p-multigrid
// solver: GLL tables, isoparametric geometry factors, line systems (the
// Def. 3.2 line blocks condensed per element segment, and their band-1
// part), transfer operators and the coarsest-level factor.  Runs once per
// problem.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace glls {

// Row-banded matrix: out[r] = sum_k coef[r*width + k] * in[start[r] + k].
struct Band1D {
    int rows = 0, cols = 0, width = 0;
    std::vector<int> start;
    std::vector<double> coef;
};

struct LevelHost {
    int dim = 2, p = 1;
    int ne[3] = {1, 1, 1};     // elements per axis
    int n[3] = {1, 1, 1};      // nodes per axis (ne * p + 1)
    long long N = 0;           // total nodes
    long long E = 0;           // total elements
    int nloc = 0;              // (p+1)^dim
    int ncomp = 0;             // geometry components: 3 (2-D) or 6 (3-D)
    std::vector<double> coords;   // [dim][N]
    std::vector<double> G;        // [ncomp][E * nloc], element-major
    std::vector<double> mass;     // [N] assembled diagonal mass
    std::vector<double> diag;     // [N] line-system diagonal (A or A~)
    std::vector<double> off[3];   // [N] line-system coupling node -> node + e_s
    std::vector<double> D;        // (p+1)^2, D[i*(p+1)+j] = pi_j'(xi_i)
    // Def. 3.2 line blocks R A_p P (GLL smoother, p >= 2), condensed per
    // element segment of each interior grid line along axis s.  Lines are
    // numbered li = (c2 - 1) * (n[o1] - 2) + (c1 - 1) over the interior
    // indices c1, c2 of the other axes o1 < o2; segment e = 0 .. ne[s]-1 holds
    // the p - 1 element-interior nodes e p + 1 .. e p + p - 1 of the line, and
    // vertex v = 1 .. ne[s]-1 is the node v p.  Task t = li * ne[s] + e.
    //   blk[s]   [ncoef][ntask]: inverse of the segment's interior block K_I
    //            (upper triangle, row-major: (p-1)p/2 values), then
    //            w_L = K_I^-1 K_{I,v=e}, then w_R = K_I^-1 K_{I,v=e+1}
    //            (zero where that vertex is a boundary node)
    //   vband[s] [nlines][ne[s]-1][2]: the Schur complement on the vertices
    //            (tridiagonal): diagonal, coupling to the next vertex
    int lblock = 0;
    std::vector<double> blk[3];
    std::vector<double> vband[3];
    Band1D P[3];                  // prolongation (this level <- level-1), per axis
    Band1D R[3];                  // restriction  (this level -> level-1), per axis
};

// Exact solver of the coarsest level: k levels of block cyclic reduction over
// the blocks of the slowest grid axis (k = 0: none), then the dense inverse of
// the remaining system.
struct CoarseHost {
    long long n = 0;                 // interior unknowns
    std::vector<long long> index;    // interior node index (level-0 grid) per unknown
    int nb = 0, m = 0;               // blocks (slowest-axis interior indices) and block size
    int cr_levels = 0;               // k
    std::vector<std::vector<double>> fh;    // per level: [kept][2][m][m]  L_i A_{i-h}^-1, U_i A_{i+h}^-1
    std::vector<std::vector<double>> agk;   // per level: [elim][3][m][m]  A_j^-1, A_j^-1 L_j, A_j^-1 U_j
    long long nr = 0;                // unknowns of the densely solved system (n when k = 0)
    std::vector<double> inv;         // its inverse, nr x nr row-major
};

std::vector<double> gll_nodes(int p, std::vector<double>* weights);
std::vector<double> derivative_matrix(int p);
std::vector<double> interpolation(int p_from, int p_to);   // [(p_to+1) x (p_from+1)]
std::vector<int> order_chain(int p_fine, bool multi_element);

// Builds all levels (index 0 = coarsest).  Returns "" on success or an error message.
// phase_ms (optional, 4 entries) accumulates the wall time of the set-up
// phases: coarse-level coordinates, geometry factors, line data (bands and
// line blocks), transfers.
std::string build_levels(int dim, const int nelem[3], int p_fine, const double* coords,
                         int smoother, int restriction, std::vector<LevelHost>& levels,
                         double* phase_ms = nullptr);
// coarse_solver: 0 automatic (block-CR depth from a cost model, 0 levels =
// dense), 1 dense A_0^-1, 2 block CR with cr_levels levels (clamped to what
// the block count allows; 0 = the model's depth, at least one level).
std::string build_coarse(const LevelHost& lv0, int coarse_solver, int cr_levels, CoarseHost& out);
int max_cr_levels(int nb);
int auto_cr_levels(int nb, int m);

}  // namespace glls
