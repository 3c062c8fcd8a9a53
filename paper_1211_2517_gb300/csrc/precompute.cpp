// Host FP64 precompute of the SVD-compressed M2L operators (Sec. 3.1).
//
//   K_fat = [K_1 ... K_316] = U Sigma [V_1^T ... V_316^T]          (Eq. (10))
//   U~ = columns of U with sigma_i >= eps sigma_0                    (Eq. (13))
//   R~ = U~  because K_o^T = K_{-o} (G radial, same surfaces), so
//        K_thin is a row-block permutation of K_fat^T (Eq. (11)) and the
//        right basis of K_thin spans the left basis of K_fat.
//   K~_o = U~^T K_o R~
//
// The SVD never forms the Gram matrix K_fat K_fat^T: singular values down
// to 1e-8 sigma_0 would drown in its rounding.  Instead:
//   1. TSQR: K_fat^T = Q R by Householder reflections, merging one n x n
//      block K_o^T at a time into a running triangular R (each worker thread
//      owns a range of offsets; the per-thread R factors are merged last).
//   2. One-sided Jacobi (Hestenes) on R: R V = W Sigma.  Since
//      K_fat = R^T Q^T = V Sigma (Q W)^T, the left singular vectors of K_fat
//      are V, accumulated from plane rotations (orthogonal to rounding).
//      Pairs are visited in a round-robin tournament so that each round's
//      n/2 rotations are independent and run in parallel.
#include <algorithm>
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>

#include "kifmm_internal.h"

namespace kifmm {

namespace {
thread_local std::string g_last_error;
constexpr double kPi = 3.14159265358979323846;
constexpr double kTieTol = 1e-13;          // equal singular values: within 1e-13 sigma_0
constexpr unsigned kCacheMagic = 0x4b4d324cu;  // "KM2L"
constexpr unsigned kCacheVersion = 4;
}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }
const char* last_error() { return g_last_error.c_str(); }

void offsets316(int (*o)[3]) {
    int k = 0;
    for (int x = -3; x <= 3; ++x)
        for (int y = -3; y <= 3; ++y)
            for (int z = -3; z <= 3; ++z) {
                int m = std::max(std::abs(x), std::max(std::abs(y), std::abs(z)));
                if (m >= 2) {
                    o[k][0] = x;
                    o[k][1] = y;
                    o[k][2] = z;
                    ++k;
                }
            }
}

namespace {
struct OffsetTable {
    int index[7 * 7 * 7];
    OffsetTable() {
        int o[kOffsets][3];
        offsets316(o);
        for (int i = 0; i < 343; ++i) index[i] = -1;
        for (int k = 0; k < kOffsets; ++k) index[(o[k][0] + 3) * 49 + (o[k][1] + 3) * 7 + (o[k][2] + 3)] = k;
    }
};
}  // namespace

int offset_index(int ox, int oy, int oz) {
    static const OffsetTable table;  // initialised once, thread-safe
    if (ox < -3 || ox > 3 || oy < -3 || oy > 3 || oz < -3 || oz > 3) return -1;
    return table.index[(ox + 3) * 49 + (oy + 3) * 7 + (oz + 3)];
}

std::vector<double> unit_surface(int p) {
    std::vector<double> u;
    u.reserve(3 * surface_count(p));
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j)
            for (int k = 0; k < p; ++k) {
                int mn = std::min(i, std::min(j, k)), mx = std::max(i, std::max(j, k));
                if (mn == 0 || mx == p - 1) {
                    u.push_back(2.0 * i / (p - 1) - 1.0);
                    u.push_back(2.0 * j / (p - 1) - 1.0);
                    u.push_back(2.0 * k / (p - 1) - 1.0);
                }
            }
    return u;
}

void unit_m2l_matrix(int p, double d, const int o[3], const std::vector<double>& u, double* K, double kh) {
    const int n = surface_count(p);
    const double s = 1.0 + d;
    for (int i = 0; i < n; ++i) {
        const double xi0 = 2.0 * o[0] + s * u[3 * i], xi1 = 2.0 * o[1] + s * u[3 * i + 1],
                     xi2 = 2.0 * o[2] + s * u[3 * i + 2];
        for (int j = 0; j < n; ++j) {
            const double a = xi0 - s * u[3 * j], b = xi1 - s * u[3 * j + 1], c = xi2 - s * u[3 * j + 2];
            const double r = std::sqrt(a * a + b * b + c * c);
            K[(size_t)i * n + j] = (kh == 0.0 ? 1.0 : std::exp(-kh * r)) / (4.0 * kPi * r);
        }
    }
}

double kernel_kh(const kifmm_m2l_params& prm) {
    return prm.kernel_id == KIFMM_KERNEL_YUKAWA ? prm.kappa * prm.box_halfwidth : 0.0;
}

int check_params(const kifmm_m2l_params* prm) {
    if (!prm) {
        set_error("params is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (prm->kernel_id != KIFMM_KERNEL_LAPLACE && prm->kernel_id != KIFMM_KERNEL_YUKAWA) {
        set_error("kernel_id " + std::to_string(prm->kernel_id) + " is not supported (0 = Laplace, 1 = Yukawa)");
        return KIFMM_ERR_UNSUPPORTED;
    }
    if (prm->kernel_id == KIFMM_KERNEL_YUKAWA &&
        !(prm->kappa > 0.0 && prm->box_halfwidth > 0.0 && std::isfinite(prm->kappa) &&
          std::isfinite(prm->box_halfwidth) && prm->kappa * prm->box_halfwidth <= 64.0)) {
        set_error("the Yukawa kernel needs kappa > 0, box_halfwidth > 0 and kappa * box_halfwidth <= 64");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (prm->p < 2 || prm->p > 12) {
        set_error("p must be in [2, 12], got " + std::to_string(prm->p));
        return KIFMM_ERR_INVALID_ARG;
    }
    if (!(prm->d >= 0.0 && prm->d <= 2.0 / 3.0)) {
        set_error("d must be in [0, 2/3]");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (!(prm->eps <= 0.0 || (prm->eps >= 1e-12 && prm->eps < 1.0)) || std::isnan(prm->eps)) {
        set_error("eps must be <= 0 (no truncation) or in [1e-12, 1)");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (prm->precision < KIFMM_PREC_FP32 || prm->precision > KIFMM_PREC_F16X3) {
        set_error("precision must be one of KIFMM_PREC_*");
        return KIFMM_ERR_INVALID_ARG;
    }
    return KIFMM_OK;
}

namespace {

// A fixed team of worker threads; run(f) calls f(tid, nthreads) on every
// member (the caller is member 0) and returns when all are done.
class ThreadTeam {
  public:
    explicit ThreadTeam(int n) : n_(n < 1 ? 1 : n) {
        for (int t = 1; t < n_; ++t) workers_.emplace_back([this, t] { loop(t); });
    }
    ~ThreadTeam() {
        {
            std::lock_guard<std::mutex> g(m_);
            stop_ = true;
            ++gen_;
        }
        cv_.notify_all();
        for (auto& w : workers_) w.join();
    }
    int size() const { return n_; }
    void run(const std::function<void(int, int)>& f) {
        {
            std::lock_guard<std::mutex> g(m_);
            job_ = &f;
            pending_ = n_ - 1;
            ++gen_;
        }
        cv_.notify_all();
        f(0, n_);
        std::unique_lock<std::mutex> lk(m_);
        done_.wait(lk, [this] { return pending_ == 0; });
        job_ = nullptr;
    }

  private:
    void loop(int t) {
        unsigned long seen = 0;
        while (true) {
            const std::function<void(int, int)>* job;
            {
                std::unique_lock<std::mutex> lk(m_);
                cv_.wait(lk, [&] { return gen_ != seen; });
                seen = gen_;
                if (stop_) return;
                job = job_;
            }
            (*job)(t, n_);
            {
                std::lock_guard<std::mutex> g(m_);
                if (--pending_ == 0) done_.notify_one();
            }
        }
    }
    int n_;
    std::vector<std::thread> workers_;
    std::mutex m_;
    std::condition_variable cv_, done_;
    const std::function<void(int, int)>* job_ = nullptr;
    unsigned long gen_ = 0;
    int pending_ = 0;
    bool stop_ = false;
};

int team_size() {
    const char* env = std::getenv("KIFMM_M2L_THREADS");
    int n = env ? std::atoi(env) : (int)std::thread::hardware_concurrency();
    if (n < 1) n = 1;
    if (n > 64) n = 64;
    return n;
}

// Dot product with eight independent partial sums: without reassociation a
// single accumulator makes every FMA wait for the previous one; eight
// chains let the loads and FMAs overlap (TSQR 1.7x faster at p = 10).
inline double dot8(const double* a, const double* b, int n) {
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0, s6 = 0, s7 = 0;
    int i = 0;
    for (; i + 8 <= n; i += 8) {
        s0 += a[i] * b[i];
        s1 += a[i + 1] * b[i + 1];
        s2 += a[i + 2] * b[i + 2];
        s3 += a[i + 3] * b[i + 3];
        s4 += a[i + 4] * b[i + 4];
        s5 += a[i + 5] * b[i + 5];
        s6 += a[i + 6] * b[i + 6];
        s7 += a[i + 7] * b[i + 7];
    }
    for (; i < n; ++i) s0 += a[i] * b[i];
    return ((s0 + s1) + (s2 + s3)) + ((s4 + s5) + (s6 + s7));
}

// Merge a dense block B (mb x n, column-major) into the upper-triangular R
// (n x n, column-major): on return R is the triangular factor of [R; B].
// B is overwritten with Householder vectors.
void householder_merge(int n, double* R, int mb, double* B) {
    for (int k = 0; k < n; ++k) {
        double* bk = B + (size_t)k * mb;
        const double xn2 = dot8(bk, bk, mb);
        if (xn2 == 0.0) continue;
        const double alpha = R[k + (size_t)k * n];
        const double beta = (alpha >= 0.0 ? -1.0 : 1.0) * std::sqrt(alpha * alpha + xn2);
        const double tau = (beta - alpha) / beta;
        const double scale = 1.0 / (alpha - beta);
        for (int i = 0; i < mb; ++i) bk[i] *= scale;
        R[k + (size_t)k * n] = beta;
        for (int c = k + 1; c < n; ++c) {
            double* bc = B + (size_t)c * mb;
            double w = R[k + (size_t)c * n] + dot8(bk, bc, mb);
            w *= tau;
            R[k + (size_t)c * n] -= w;
            for (int i = 0; i < mb; ++i) bc[i] -= w * bk[i];
        }
    }
}

// Triangular factor of K_fat^T (316 n x n).  Returns R, column-major n x n.
std::vector<double> tsqr_kfat_t(int p, double d, double kh, const std::vector<double>& u, ThreadTeam& team) {
    const int n = surface_count(p);
    int offs[kOffsets][3];
    offsets316(offs);
    const int nthreads = team.size();
    std::vector<std::vector<double>> Rt(nthreads, std::vector<double>((size_t)n * n, 0.0));
    team.run([&](int tid, int) {
        std::vector<double> K((size_t)n * n), B((size_t)n * n);
        const int lo = (int)((long)kOffsets * tid / nthreads), hi = (int)((long)kOffsets * (tid + 1) / nthreads);
        for (int k = lo; k < hi; ++k) {
            unit_m2l_matrix(p, d, offs[k], u, K.data(), kh);
            // block of K_fat^T: rows j (source points), columns i; B(j,i) = K_o[i][j]
            // column-major B: column i contiguous over j -> B[i*n + j] = K[i*n + j]
            std::copy(K.begin(), K.end(), B.begin());
            householder_merge(n, Rt[tid].data(), n, B.data());
        }
    });
    std::vector<double> R = Rt[0];
    for (int t = 1; t < nthreads; ++t) householder_merge(n, R.data(), n, Rt[t].data());
    return R;
}

// One-sided Jacobi on A (n x n column-major, n even).  On return V holds
// the right singular vectors (column-major) and sig the singular values,
// both sorted by descending singular value; when AV is given it receives
// the rotated columns A v_j = sigma_j u_j in the same order.
void jacobi_svd(int n, std::vector<double>& A, std::vector<double>& V, std::vector<double>& sig, ThreadTeam& team,
                std::vector<double>* AV = nullptr) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[i + (size_t)i * n] = 1.0;
    const double tol = 1e-15;
    // round-robin tournament: player 0 fixed, others rotate
    std::vector<int> ring(n);
    std::iota(ring.begin(), ring.end(), 0);
    std::vector<long> rot_count(team.size());
    for (int sweep = 0; sweep < 80; ++sweep) {
        long rotations = 0;
        std::fill(rot_count.begin(), rot_count.end(), 0L);
        for (int round = 0; round < n - 1; ++round) {
          team.run([&](int tid, int nt) {
            for (int m = tid; m < n / 2; m += nt) {
                int a = ring[m], b = ring[n - 1 - m];
                if (a > b) std::swap(a, b);
                double* ap = A.data() + (size_t)a * n;
                double* aq = A.data() + (size_t)b * n;
                const double alpha = dot8(ap, ap, n), beta = dot8(aq, aq, n), gamma = dot8(ap, aq, n);
                if (gamma == 0.0 || std::fabs(gamma) <= tol * std::sqrt(alpha * beta)) continue;
                const double zeta = (beta - alpha) / (2.0 * gamma);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                for (int i = 0; i < n; ++i) {
                    const double x = ap[i], y = aq[i];
                    ap[i] = c * x - s * y;
                    aq[i] = s * x + c * y;
                }
                double* vp = V.data() + (size_t)a * n;
                double* vq = V.data() + (size_t)b * n;
                for (int i = 0; i < n; ++i) {
                    const double x = vp[i], y = vq[i];
                    vp[i] = c * x - s * y;
                    vq[i] = s * x + c * y;
                }
                ++rot_count[tid];
            }
          });
            // rotate positions 1..n-1
            int last = ring[n - 1];
            for (int i = n - 1; i > 1; --i) ring[i] = ring[i - 1];
            ring[1] = last;
        }
        for (long c : rot_count) rotations += c;
        if (rotations == 0) break;
    }
    std::vector<double> s(n);
    for (int j = 0; j < n; ++j) {
        double acc = 0;
        const double* aj = A.data() + (size_t)j * n;
        for (int i = 0; i < n; ++i) acc += aj[i] * aj[i];
        s[j] = std::sqrt(acc);
    }
    std::vector<int> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return s[x] > s[y]; });
    std::vector<double> Vs((size_t)n * n);
    sig.resize(n);
    if (AV) AV->resize((size_t)n * n);
    for (int j = 0; j < n; ++j) {
        sig[j] = s[ord[j]];
        std::copy(V.begin() + (size_t)ord[j] * n, V.begin() + (size_t)(ord[j] + 1) * n, Vs.begin() + (size_t)j * n);
        if (AV)
            std::copy(A.begin() + (size_t)ord[j] * n, A.begin() + (size_t)(ord[j] + 1) * n,
                      AV->begin() + (size_t)j * n);
    }
    V.swap(Vs);
}

// Right singular vectors and singular values of A (n x n column-major) by the
// preconditioned one-sided Jacobi method of Drmac and Veselic (SIAM J. Matrix
// Anal. Appl. 29, 2008): A P = Q R1 by Householder QR with column pivoting,
// then one-sided Jacobi on the columns of R1^T, which are graded, so the
// sweeps converge several times sooner than on A itself (14 against 40 for
// the K_fat factor at p = 10).  With R1^T Y = X S the right singular vectors
// of A are P X (X the normalised columns): no rotation is accumulated.  A is
// overwritten; V column-major, both sorted by descending singular value.
void jacobi_svd_pre(int n, std::vector<double>& A, std::vector<double>& V, std::vector<double>& sig, ThreadTeam& team) {
    std::vector<int> perm(n);
    std::iota(perm.begin(), perm.end(), 0);
    std::vector<double> cn(n), cn0(n);
    for (int j = 0; j < n; ++j) {
        double acc = 0;
        const double* aj = A.data() + (size_t)j * n;
        for (int i = 0; i < n; ++i) acc += aj[i] * aj[i];
        cn[j] = cn0[j] = acc;
    }
    std::vector<double> v(n);
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int j = k + 1; j < n; ++j) if (cn[j] > cn[piv]) piv = j;
        if (piv != k) {
            std::swap_ranges(A.begin() + (size_t)k * n, A.begin() + (size_t)(k + 1) * n, A.begin() + (size_t)piv * n);
            std::swap(cn[k], cn[piv]); std::swap(cn0[k], cn0[piv]); std::swap(perm[k], perm[piv]);
        }
        double* ak = A.data() + (size_t)k * n;
        const double nrm = std::sqrt(dot8(ak + k, ak + k, n - k));
        if (nrm == 0.0) continue;
        const double alpha = ak[k] > 0 ? -nrm : nrm;
        // v = x - alpha e1, normalised so that H = I - 2 v v^T / (v^T v)
        for (int i = k; i < n; ++i) v[i] = ak[i];
        v[k] -= alpha;
        const double vv = dot8(v.data() + k, v.data() + k, n - k);
        ak[k] = alpha;
        for (int i = k + 1; i < n; ++i) ak[i] = 0.0;
        if (vv == 0.0) continue;
        team.run([&](int tid, int nt) {
            for (int j = k + 1 + tid; j < n; j += nt) {
                double* aj = A.data() + (size_t)j * n;
                const double d = dot8(v.data() + k, aj + k, n - k);
                const double w = 2.0 * d / vv;
                for (int i = k; i < n; ++i) aj[i] -= w * v[i];
            }
        });
        for (int j = k + 1; j < n; ++j) {
            const double* aj = A.data() + (size_t)j * n;
            cn[j] -= aj[k] * aj[k];
            if (cn[j] < 1e-8 * cn0[j]) {  // recompute after cancellation
                double acc = 0;
                for (int i = k + 1; i < n; ++i) acc += aj[i] * aj[i];
                cn[j] = cn0[j] = acc;
            }
        }
    }
    // B = R1^T (column j of B = row j of R1), column-major
    std::vector<double> B((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i <= j; ++i) B[(size_t)i * n + j] = A[(size_t)j * n + i];
    const double tol = 1e-15;
    std::vector<int> ring(n);
    std::iota(ring.begin(), ring.end(), 0);
    std::vector<long> rot_count(team.size());
    for (int sweep = 0; sweep < 80; ++sweep) {
        std::fill(rot_count.begin(), rot_count.end(), 0L);
        for (int round = 0; round < n - 1; ++round) {
            team.run([&](int tid, int nt) {
                for (int m = tid; m < n / 2; m += nt) {
                    int a = ring[m], b = ring[n - 1 - m];
                    if (a > b) std::swap(a, b);
                    double* ap = B.data() + (size_t)a * n;
                    double* aq = B.data() + (size_t)b * n;
                    const double al = dot8(ap, ap, n), be = dot8(aq, aq, n), ga = dot8(ap, aq, n);
                    if (ga == 0.0 || std::fabs(ga) <= tol * std::sqrt(al * be)) continue;
                    const double zeta = (be - al) / (2.0 * ga);
                    const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                    const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
                    for (int i = 0; i < n; ++i) { const double x = ap[i], y = aq[i]; ap[i] = c * x - sn * y; aq[i] = sn * x + c * y; }
                    ++rot_count[tid];
                }
            });
            int last = ring[n - 1];
            for (int i = n - 1; i > 1; --i) ring[i] = ring[i - 1];
            ring[1] = last;
        }
        long rotations = 0;
        for (long c : rot_count) rotations += c;
        if (rotations == 0) break;
    }
    std::vector<double> s(n);
    for (int j = 0; j < n; ++j) {
        double acc = 0;
        const double* bj = B.data() + (size_t)j * n;
        for (int i = 0; i < n; ++i) acc += bj[i] * bj[i];
        s[j] = std::sqrt(acc);
    }
    std::vector<int> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return s[x] > s[y]; });
    sig.resize(n);
    V.assign((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        const int src = ord[j];
        sig[j] = s[src];
        const double* bj = B.data() + (size_t)src * n;
        double* vj = V.data() + (size_t)j * n;
        if (s[src] > 0)
            for (int k = 0; k < n; ++k) vj[perm[k]] = bj[k] / s[src];
    }
}

int truncation_rank(const std::vector<double>& sig, double eps) {
    const int n = (int)sig.size();
    if (eps <= 0) return n;
    int r = 0;
    while (r < n && sig[r] >= eps * sig[0]) ++r;
    while (r > 0 && r < n && sig[r - 1] - sig[r] <= kTieTol * sig[0]) ++r;
    return r;
}

std::string cache_path(const kifmm_m2l_params& prm) {
    const char* dir = std::getenv("KIFMM_M2L_CACHE");
    if (!dir || !*dir) return std::string();
    char name[256];
    std::snprintf(name, sizeof(name), "/kifmm_m2l_v%u_k%d_p%d_d%.17g_eps%.17g_kh%.17g.bin", kCacheVersion,
                  prm.kernel_id, prm.p, prm.d, prm.eps, kernel_kh(prm));
    return std::string(dir) + name;
}

bool load_cache(const std::string& path, const kifmm_m2l_params& prm, Factors& f) {
    if (path.empty()) return false;
    FILE* fp = std::fopen(path.c_str(), "rb");
    if (!fp) return false;
    unsigned hdr[2];
    int dims[4];
    double pd[3];
    bool ok = std::fread(hdr, sizeof(hdr), 1, fp) == 1 && hdr[0] == kCacheMagic && hdr[1] == kCacheVersion &&
              std::fread(dims, sizeof(dims), 1, fp) == 1 && std::fread(pd, sizeof(pd), 1, fp) == 1 &&
              dims[0] == prm.kernel_id && dims[1] == prm.p && pd[0] == prm.d && pd[1] == prm.eps &&
              pd[2] == kernel_kh(prm);
    if (ok) {
        f.p = dims[1];
        f.n = surface_count(f.p);
        f.r = dims[2];
        ok = dims[3] == f.n && f.r >= 1 && f.r <= f.n;
    }
    if (ok) {
        f.d = prm.d;
        f.eps = prm.eps;
        f.sigma.resize(f.n);
        f.U.resize((size_t)f.n * f.r);
        f.C.resize((size_t)kOffsets * f.r * f.r);
        ok = std::fread(f.sigma.data(), sizeof(double), f.n, fp) == (size_t)f.n &&
             std::fread(f.U.data(), sizeof(double), f.U.size(), fp) == f.U.size() &&
             std::fread(f.C.data(), sizeof(double), f.C.size(), fp) == f.C.size() &&
             std::fread(&f.sym_err, sizeof(double), 1, fp) == 1;
    }
    std::fclose(fp);
    return ok;
}

void store_cache(const std::string& path, const kifmm_m2l_params& prm, const Factors& f) {
    if (path.empty()) return;
    std::string tmp = path + ".tmp" + std::to_string((long)std::rand());
    FILE* fp = std::fopen(tmp.c_str(), "wb");
    if (!fp) return;
    unsigned hdr[2] = {kCacheMagic, kCacheVersion};
    int dims[4] = {prm.kernel_id, prm.p, f.r, f.n};
    double pd[3] = {prm.d, prm.eps, kernel_kh(prm)};
    bool ok = std::fwrite(hdr, sizeof(hdr), 1, fp) == 1 && std::fwrite(dims, sizeof(dims), 1, fp) == 1 &&
              std::fwrite(pd, sizeof(pd), 1, fp) == 1 &&
              std::fwrite(f.sigma.data(), sizeof(double), f.n, fp) == (size_t)f.n &&
              std::fwrite(f.U.data(), sizeof(double), f.U.size(), fp) == f.U.size() &&
              std::fwrite(f.C.data(), sizeof(double), f.C.size(), fp) == f.C.size() &&
              std::fwrite(&f.sym_err, sizeof(double), 1, fp) == 1;
    ok = (std::fclose(fp) == 0) && ok;
    if (ok)
        std::rename(tmp.c_str(), path.c_str());
    else
        std::remove(tmp.c_str());
}

}  // namespace

namespace {

// The factors of the last precompute in this process (one entry, held until
// exit): a size query followed by the data query, or several plans of one
// operator, cost one precompute.
struct Memo {
    bool valid = false;
    int kernel_id = 0, p = 0;
    double d = 0, eps = 0, kh = 0;
    Factors f;
};
std::mutex g_memo_mutex;
Memo g_memo;

bool memo_matches(const kifmm_m2l_params& prm) {
    return g_memo.valid && g_memo.kernel_id == prm.kernel_id && g_memo.p == prm.p && g_memo.d == prm.d &&
           g_memo.eps == prm.eps && g_memo.kh == kernel_kh(prm);
}

}  // namespace

int compute_factors(const kifmm_m2l_params& prm, Factors& f) {
    int st = check_params(&prm);
    if (st != KIFMM_OK) return st;
    try {
        std::lock_guard<std::mutex> lock(g_memo_mutex);
        if (memo_matches(prm)) {
            f = g_memo.f;
            return KIFMM_OK;
        }
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed copying the factors");
        return KIFMM_ERR_OOM;
    }
    st = compute_factors_uncached(prm, f);
    if (st != KIFMM_OK) return st;
    try {
        std::lock_guard<std::mutex> lock(g_memo_mutex);
        g_memo.valid = false;
        g_memo.f = f;
        g_memo.kernel_id = prm.kernel_id;
        g_memo.p = prm.p;
        g_memo.d = prm.d;
        g_memo.eps = prm.eps;
        g_memo.kh = kernel_kh(prm);
        g_memo.valid = true;
    } catch (const std::bad_alloc&) {
        g_memo.valid = false;  // the factors are returned all the same
    }
    return KIFMM_OK;
}

int compute_factors_uncached(const kifmm_m2l_params& prm, Factors& f) {
    int st = check_params(&prm);
    if (st != KIFMM_OK) return st;
    const std::string cpath = cache_path(prm);
    if (load_cache(cpath, prm, f)) return KIFMM_OK;

    const int p = prm.p, n = surface_count(p);
    const std::vector<double> u = unit_surface(p);
    try {
        ThreadTeam team(team_size());
        std::vector<double> R = tsqr_kfat_t(p, prm.d, kernel_kh(prm), u, team);
        // zero the strict lower triangle (Householder vectors are not stored in R)
        for (int c = 0; c < n; ++c)
            for (int i = c + 1; i < n; ++i) R[i + (size_t)c * n] = 0.0;
        std::vector<double> V, sig;
        jacobi_svd_pre(n, R, V, sig, team);
        const int r = truncation_rank(sig, prm.eps);

        f.p = p;
        f.n = n;
        f.r = r;
        f.d = prm.d;
        f.eps = prm.eps;
        f.sigma = sig;
        f.U.assign((size_t)n * r, 0.0);
        for (int j = 0; j < r; ++j) {
            // sign rule: the largest-magnitude entry of each column is positive
            const double* vj = V.data() + (size_t)j * n;
            int imax = 0;
            for (int i = 1; i < n; ++i)
                if (std::fabs(vj[i]) > std::fabs(vj[imax])) imax = i;
            const double sgn = vj[imax] < 0 ? -1.0 : 1.0;
            for (int i = 0; i < n; ++i) f.U[(size_t)i * r + j] = sgn * vj[i];
        }

        // cores K~_o = U~^T K_o U~.  K_o^T = K_{-o} (G radial, one point
        // pattern for both surfaces), so K~_{-o} = K~_o^T: one core of every
        // (o, -o) pair is formed, plus every 40th partner as a check of the
        // identity the transposes rely on
        int offs[kOffsets][3];
        offsets316(offs);
        std::vector<int> partner(kOffsets), formed;
        for (int k = 0; k < kOffsets; ++k) partner[k] = offset_index(-offs[k][0], -offs[k][1], -offs[k][2]);
        for (int k = 0; k < kOffsets; ++k)
            if (k < partner[k] || k % 40 == 0) formed.push_back(k);
        f.C.assign((size_t)kOffsets * r * r, 0.0);
        team.run([&](int tid, int nt) {
            std::vector<double> K((size_t)n * n), T((size_t)n * r);
            for (size_t fi = tid; fi < formed.size(); fi += nt) {
                const int k = formed[fi];
                unit_m2l_matrix(p, prm.d, offs[k], u, K.data(), kernel_kh(prm));
                // T = K_o U~  (n x r)
                std::fill(T.begin(), T.end(), 0.0);
                for (int i = 0; i < n; ++i) {
                    double* ti = T.data() + (size_t)i * r;
                    const double* ki = K.data() + (size_t)i * n;
                    for (int j = 0; j < n; ++j) {
                        const double kij = ki[j];
                        const double* uj = f.U.data() + (size_t)j * r;
                        for (int b = 0; b < r; ++b) ti[b] += kij * uj[b];
                    }
                }
                // C = U~^T T  (r x r)
                double* ck = f.C.data() + (size_t)k * r * r;
                for (int i = 0; i < n; ++i) {
                    const double* ui = f.U.data() + (size_t)i * r;
                    const double* ti = T.data() + (size_t)i * r;
                    for (int a = 0; a < r; ++a) {
                        const double uia = ui[a];
                        double* ca = ck + (size_t)a * r;
                        for (int b = 0; b < r; ++b) ca[b] += uia * ti[b];
                    }
                }
            }
        });
        // symmetry K~_o^T = K~_{-o} on the pairs formed both ways, then the
        // transposes for the rest
        double cmax = 0, dmax = 0;
        for (int k : formed) {
            const int km = partner[k];
            if (k < km && km % 40 != 0) continue;
            const double* ck = f.C.data() + (size_t)k * r * r;
            const double* cm = f.C.data() + (size_t)km * r * r;
            for (int a = 0; a < r; ++a)
                for (int b = 0; b < r; ++b) {
                    cmax = std::max(cmax, std::fabs(ck[(size_t)a * r + b]));
                    dmax = std::max(dmax, std::fabs(ck[(size_t)a * r + b] - cm[(size_t)b * r + a]));
                }
        }
        f.sym_err = cmax > 0 ? dmax / cmax : 0.0;
        for (int k = 0; k < kOffsets; ++k) {
            if (k < partner[k] || k % 40 == 0) continue;
            const double* cp = f.C.data() + (size_t)partner[k] * r * r;
            double* ck = f.C.data() + (size_t)k * r * r;
            for (int a = 0; a < r; ++a)
                for (int b = 0; b < r; ++b) ck[(size_t)a * r + b] = cp[(size_t)b * r + a];
        }
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed in the FP64 precompute");
        return KIFMM_ERR_OOM;
    }
    store_cache(cpath, prm, f);
    return KIFMM_OK;
}

int compute_stage2(const Factors& f, double c2, Stage2& s2) {
    if (!(c2 > 0) || f.r < 1 || f.sigma.empty()) {
        set_error("stage 2 needs c2 > 0 and computed factors");
        return KIFMM_ERR_INVALID_ARG;
    }
    const int r = f.r;
    s2.c2 = c2;
    s2.eps2 = c2 * (f.eps > 0 ? f.eps : 0.0) / r;
    const double thr = s2.eps2 * f.sigma[0];
    s2.k.assign(kOffsets, 0);
    s2.Uh.assign(kOffsets, {});
    s2.Vh.assign(kOffsets, {});
    try {
        ThreadTeam team(team_size());
        team.run([&](int tid, int nt) {
            ThreadTeam solo(1);
            // the round-robin Jacobi pairs columns two by two: pad an odd r with
            // a zero row and column (one extra zero singular value)
            const int re = r + (r & 1);
            std::vector<double> A, V, sig, u(r);
            for (int o = tid; o < kOffsets; o += nt) {
                const double* C = f.C.data() + (size_t)o * r * r;
                // columns of K~_o, column-major, for the one-sided Jacobi SVD
                A.assign((size_t)re * re, 0.0);
                for (int c = 0; c < r; ++c)
                    for (int i = 0; i < r; ++i) A[(size_t)c * re + i] = C[(size_t)i * r + c];
                jacobi_svd_pre(re, A, V, sig, solo);  // V: right singular vectors q_j (columns), sig descending
                int k = 0;
                while (k < r && sig[k] >= thr && sig[k] > 0) ++k;
                s2.k[o] = k;
                s2.Uh[o].assign((size_t)r * k, 0.0);
                s2.Vh[o].assign((size_t)k * r, 0.0);
                for (int j = 0; j < k; ++j) {
                    const double* q = V.data() + (size_t)j * re;
                    // u_j = K~_o q_j / sigma_j
                    for (int a = 0; a < r; ++a) u[a] = dot8(C + (size_t)a * r, q, r) / sig[j];
                    for (int a = 0; a < r; ++a) s2.Uh[o][(size_t)a * k + j] = u[a];
                    for (int b = 0; b < r; ++b) s2.Vh[o][(size_t)j * r + b] = sig[j] * q[b];
                }
            }
        });
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed in the stage-2 precompute");
        return KIFMM_ERR_OOM;
    }
    return KIFMM_OK;
}

int compute_pass_ops(int p, double d, int r, const std::vector<double>& U, double rcond, PassOps& out) {
    const int n = surface_count(p);
    if (r < 1 || (int)U.size() != n * r || !(rcond > 0) || !(rcond < 1)) {
        set_error("pass operators need the stage-1 basis and 0 < rcond < 1");
        return KIFMM_ERR_INVALID_ARG;
    }
    const std::vector<double> u = unit_surface(p);
    constexpr double kInv4Pi = 0.07957747154594767;  // 1 / (4 pi)
    auto G = [&](const double* x, const double* y) {
        const double a = x[0] - y[0], b = x[1] - y[1], c = x[2] - y[2];
        return kInv4Pi / std::sqrt(a * a + b * b + c * c);
    };
    try {
        ThreadTeam team(team_size());
        // upward check surface x^u ((3-2d) u) and equivalent surface y^u ((1+d) u) of a unit box
        std::vector<double> xu((size_t)3 * n), yu((size_t)3 * n);
        for (int i = 0; i < 3 * n; ++i) {
            xu[i] = (3.0 - 2.0 * d) * u[i];
            yu[i] = (1.0 + d) * u[i];
        }
        // A = K(x^u, y^u), column-major
        std::vector<double> A((size_t)n * n), V, sig, AV;
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) A[(size_t)j * n + i] = G(&xu[3 * i], &yu[3 * j]);
        jacobi_svd(n, A, V, sig, team, &AV);
        int kept = 0;
        while (kept < n && sig[kept] >= rcond * sig[0] && sig[kept] > 0) ++kept;
        // E_u = pinv(A) = sum_k v_k (A v_k)^T / sigma_k^2, row-major [n][n]
        std::vector<double> E((size_t)n * n, 0.0);
        team.run([&](int tid, int nt) {
            for (int i = tid; i < n; i += nt) {
                double* ei = E.data() + (size_t)i * n;
                for (int k = 0; k < kept; ++k) {
                    const double w = V[(size_t)k * n + i] / (sig[k] * sig[k]);
                    const double* ak = AV.data() + (size_t)k * n;
                    for (int j = 0; j < n; ++j) ei[j] += w * ak[j];
                }
            }
        });
        // Ws = U~^T E_u  [r][n]
        out.Ws.assign((size_t)r * n, 0.0);
        team.run([&](int tid, int nt) {
            for (int a = tid; a < r; a += nt) {
                double* wa = out.Ws.data() + (size_t)a * n;
                for (int i = 0; i < n; ++i) {
                    const double uia = U[(size_t)i * r + a];
                    const double* ei = E.data() + (size_t)i * n;
                    for (int j = 0; j < n; ++j) wa[j] += uia * ei[j];
                }
            }
        });
        // Mt[c] = U~^T E_u K(x^u, y^u of child c) U~ = Ws K_c U~; child c of a
        // unit parent: centre (2 b - 1) / 2 with c = 4 b_x + 2 b_y + b_z,
        // half-width 1/2
        out.Mt.assign((size_t)8 * r * r, 0.0);
        team.run([&](int tid, int nt) {
            std::vector<double> yc((size_t)3 * n), T((size_t)r * n);
            for (int c = tid; c < 8; c += nt) {
                const double ctr[3] = {((c >> 2) & 1) - 0.5, ((c >> 1) & 1) - 0.5, (c & 1) - 0.5};
                for (int j = 0; j < n; ++j)
                    for (int t = 0; t < 3; ++t) yc[3 * j + t] = ctr[t] + 0.5 * (1.0 + d) * u[3 * j + t];
                // T = Ws K_c  [r][n]
                std::fill(T.begin(), T.end(), 0.0);
                for (int i = 0; i < n; ++i)
                    for (int j = 0; j < n; ++j) {
                        const double kij = G(&xu[3 * i], &yc[3 * j]);
                        for (int a = 0; a < r; ++a) T[(size_t)a * n + j] += out.Ws[(size_t)a * n + i] * kij;
                    }
                double* m = out.Mt.data() + (size_t)c * r * r;
                for (int a = 0; a < r; ++a)
                    for (int j = 0; j < n; ++j) {
                        const double taj = T[(size_t)a * n + j];
                        const double* uj = U.data() + (size_t)j * r;
                        for (int b = 0; b < r; ++b) m[(size_t)a * r + b] += taj * uj[b];
                    }
            }
        });
        out.rcond = rcond;
        out.kept = kept;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed in the pass-operator precompute");
        return KIFMM_ERR_OOM;
    }
    return KIFMM_OK;
}

int build_pairs(int level, int n_boxes, const int32_t* ijk, std::vector<int32_t>& tgt, std::vector<int32_t>& src,
                std::vector<int32_t>& off) {
    tgt.clear();
    src.clear();
    off.clear();
    if (level < 0 || level > 20 || n_boxes < 0 || (n_boxes > 0 && !ijk)) {
        set_error("invalid level / n_boxes / box_ijk");
        return KIFMM_ERR_INVALID_ARG;
    }
    const int64_t m = int64_t(1) << level;
    std::vector<std::pair<int64_t, int32_t>> keys(n_boxes);
    for (int b = 0; b < n_boxes; ++b) {
        const int64_t x = ijk[3 * b], y = ijk[3 * b + 1], z = ijk[3 * b + 2];
        if (x < 0 || y < 0 || z < 0 || x >= m || y >= m || z >= m) {
            set_error("box " + std::to_string(b) + " has coordinates outside [0, 2^level)");
            return KIFMM_ERR_INVALID_ARG;
        }
        keys[b] = {(x << 42) | (y << 21) | z, b};
    }
    std::sort(keys.begin(), keys.end());
    for (int b = 1; b < n_boxes; ++b)
        if (keys[b].first == keys[b - 1].first) {
            set_error("duplicate box coordinates");
            return KIFMM_ERR_INVALID_ARG;
        }
    auto find = [&](int64_t x, int64_t y, int64_t z) -> int32_t {
        if (x < 0 || y < 0 || z < 0 || x >= m || y >= m || z >= m) return -1;
        const int64_t key = (x << 42) | (y << 21) | z;
        auto it = std::lower_bound(keys.begin(), keys.end(), std::make_pair(key, (int32_t)-1));
        return (it != keys.end() && it->first == key) ? it->second : -1;
    };
    // per offset buckets (offset-major order), each bucket in target order
    std::vector<std::vector<std::pair<int32_t, int32_t>>> bucket(kOffsets);
    for (int t = 0; t < n_boxes; ++t) {
        const int64_t tx = ijk[3 * t], ty = ijk[3 * t + 1], tz = ijk[3 * t + 2];
        const int64_t px = tx >> 1, py = ty >> 1, pz = tz >> 1;
        // children of the parent's near-field boxes (Sec. 2.1), minus t's near field
        for (int64_t sx = 2 * px - 2; sx <= 2 * px + 3; ++sx)
            for (int64_t sy = 2 * py - 2; sy <= 2 * py + 3; ++sy)
                for (int64_t sz = 2 * pz - 2; sz <= 2 * pz + 3; ++sz) {
                    const int64_t ox = tx - sx, oy = ty - sy, oz = tz - sz;
                    if (std::max(std::llabs(ox), std::max(std::llabs(oy), std::llabs(oz))) <= 1) continue;
                    const int32_t s = find(sx, sy, sz);
                    if (s < 0) continue;
                    bucket[offset_index((int)ox, (int)oy, (int)oz)].push_back({t, s});
                }
    }
    size_t total = 0;
    for (auto& b : bucket) total += b.size();
    tgt.reserve(total);
    src.reserve(total);
    off.reserve(total);
    for (int k = 0; k < kOffsets; ++k)
        for (auto& ts : bucket[k]) {
            tgt.push_back(ts.first);
            src.push_back(ts.second);
            off.push_back(k);
        }
    return KIFMM_OK;
}

}  // namespace kifmm
