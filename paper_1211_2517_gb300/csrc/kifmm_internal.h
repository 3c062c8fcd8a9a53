// Internal declarations shared by the host precompute, the plan and the
// kernels.  Not part of the public ABI (see include/kifmm_m2l.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "kifmm_m2l.h"

namespace kifmm {

constexpr int kOffsets = KIFMM_N_OFFSETS;

// Thread-local last-error message behind kifmm_m2l_last_error().
void set_error(const std::string& msg);
const char* last_error();

// Number of surface points for p points per edge: 6(p-1)^2 + 2.
inline int surface_count(int p) { return 6 * (p - 1) * (p - 1) + 2; }

// The 316 offsets o in {-3..3}^3 with max|o_i| >= 2, lexicographic.
void offsets316(int (*o)[3]);
// Index of offset o in offsets316(), or -1.
int offset_index(int ox, int oy, int oz);

// Points of the [-1,1]^3 cube boundary (lexicographic grid order), [n][3].
std::vector<double> unit_surface(int p);

// Entry (i, j) of the unit-level translation matrix K_o (Sec. 2.2 Eq. (4),
// surfaces of Sec. 2.1): g(|2 o + (1+d)(u_i - u_j)|) with g(r) = exp(-kh r) /
// (4 pi r); kh = 0 is the Laplace kernel, kh = kappa h the Yukawa kernel at
// box half-width h (times h).
void unit_m2l_matrix(int p, double d, const int o[3], const std::vector<double>& u, double* K, double kh = 0.0);

// kappa h of a plan's kernel (0 for the Laplace kernel).
double kernel_kh(const kifmm_m2l_params& prm);

// FP64 factors of the stage-1 compression (Sec. 3.1).
struct Factors {
    int p = 0, n = 0, r = 0;
    double d = 0, eps = 0;
    std::vector<double> sigma;  // [n] singular values of K_fat, descending
    std::vector<double> U;      // [n][r] row-major, U~ (= R~)
    std::vector<double> C;      // [316][r][r] row-major, K~_o = U~^T K_o U~
    double sym_err = 0;         // max |K~_o^T - K~_{-o}| / max |K~|
};

// Full host precompute, with the optional on-disk cache and a one-entry
// in-process memo of the last result.  Returns a status.
int compute_factors(const kifmm_m2l_params& prm, Factors& f);
// The same without the in-process memo.
int compute_factors_uncached(const kifmm_m2l_params& prm, Factors& f);

// Stage-2 per-offset factors (Sec. 3.2, Eq. (17)): K~_o = U_o S_o Q_o^T,
// keep the k_o singular values >= eps2 * sigma_0(K_fat) with
// eps2 = c2 * eps1 / r (Eq. (18)); Uhat_o = U_o[:, :k_o] (r x k_o),
// Vhat_o = S Q^T restricted to those k_o (k_o x r), both row-major.
struct Stage2 {
    double c2 = 0, eps2 = 0;
    std::vector<int> k;                   // [316]
    std::vector<std::vector<double>> Uh;  // [316] r x k_o
    std::vector<std::vector<double>> Vh;  // [316] k_o x r
};
int compute_stage2(const Factors& f, double c2, Stage2& s2);

// Compressed pass operators of Sec. 3.3 for a unit parent box, with the
// basis U (n x r row-major) serving as both R~ and U~:
//   Ws    = U~^T E_u                (r x n)   S~ of a leaf of half-width h is h Ws K(x^u, points)
//   Mt[c] = U~^T E_u K(x^u, y^u_c) U~  (r x r)   M~ of the child in octant c
// E_u is the pseudo-inverse of K(x^u, y^u) keeping the singular values
// >= rcond * sigma_0 (their count in `kept`); octant c = 4 b_x + 2 b_y + b_z
// puts the child's centre at (2 b - 1) / 2.  The downward operators are the
// transposes: the downward check / equivalent surfaces are the upward
// equivalent / check ones (Sec. 2.1), so K(x^d, y^d) = K(x^u, y^u)^T and
// T~'s factor E_d U~ = Ws^T, L~_c = Mt[c]^T.
struct PassOps {
    double rcond = 0;
    int kept = 0;
    std::vector<double> Ws;  // [r][n]
    std::vector<double> Mt;  // [8][r][r]
};
int compute_pass_ops(int p, double d, int r, const std::vector<double>& U, double rcond, PassOps& out);

// Validate a params struct; returns a status and sets the error message.
int check_params(const kifmm_m2l_params* prm);

// Interaction-list pairs of one level (Sec. 2.1), sorted by (offset, target).
// Returns a status.
int build_pairs(int level, int n_boxes, const int32_t* ijk, std::vector<int32_t>& tgt,
                std::vector<int32_t>& src, std::vector<int32_t>& off);

}  // namespace kifmm
