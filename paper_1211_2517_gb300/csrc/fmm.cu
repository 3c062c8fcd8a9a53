// Point-source evaluation (include/kifmm_m2l.h, kifmm_fmm_*): the complete
// algorithm of Sec. 4 for point sources, with the compressed upward and
// downward passes of Sec. 3.3.
//
// Host, once per tree: a uniform-depth octree (points sorted by the Morton
// key of their leaf, the non-empty boxes of every level, parents and
// octants, the near leaves of every leaf), the M2L interaction state of
// levels 2..depth registered on the plan under a reserved instance, and the
// row tables of the M~ and L~ gathers (children grouped by octant, 128 rows
// per tile).
//
// Device, per evaluate, in stream order:
//   gather     densities into the leaf-ordered point array        (CUDA cores)
//   S~         q~_leaf = sum_j q_j s_j over the leaf's points, s_j the
//              point's compressed row (below)                      (CUDA cores)
//   M~         level by level, children -> parents: gather GEMM over the
//              8 octant groups with FP32 reductions, then split   (tensor cores)
//   M2L        the plan's core over every level's pairs           (tensor cores)
//   L~         level by level, parents -> children: split of the
//              parents' p~, gather GEMM adding into the children  (tensor cores)
//   leaf sums  far field t_i . p~_leaf (T~ and L2T in one dot product per
//              point) plus the near field (double layer: dG/dn(y)), in the
//              caller's order                                      (CUDA cores)
//
// The per-point rows are formed once per tree (and per set of normals) in
// FP64 from the FP64 S~ factor Ws and stored in FP32: t(s) = 1/(4 pi) Ws g(s)
// with g_i = 1 / |x_i - s| over the check points x_i of the leaf (leaf
// units), which is both the T~ row (far field at s) and, since the upward
// check surface is the downward equivalent surface and G is symmetric, the
// S~ row of a unit charge at s; dipoles get their own S~ rows from
// n . (x_i - y) / |x_i - y|^3 (Eq. (26)).  Ws carries the pseudo-inverse
// cutoff's large entries; forming the rows in FP64 keeps that amplification
// out of the FP32 evaluation, which then sees well-conditioned r-vectors.
//
// Layout (rows = boxes of levels 2..depth back to back, level order):
//   qb3  BF16 [3][rows + 1][rp]  q~ pieces, last row zero
//   pt   FP32 [rows][rp]         p~
//   qf   FP32 [rows][rp]          q~ of every level (M~ accumulates into it)
//   qh, qs  f16x3 plans: the core's FP16 pieces [2][rows + 1][rp] of qf, row factors
//   sl   BF16 [3][(tiles + 1) * 128][rp]   one level's p~ pieces (L~ input)
//   trows, drows  FP32 [points][rp]  the per-point T~ rows and the dipoles' S~ rows
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "kernels.h"
#include "kifmm_internal.h"
#include "plan.h"

using namespace kifmm;

namespace {

// Pseudo-inverse cutoff of the check-to-equivalent solves (relative to the
// largest singular value).
constexpr double kPassRcond = 1e-9;

uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1FFFFF;
    x = (x | (x << 32)) & 0x1F00000000FFFFull;
    x = (x | (x << 16)) & 0x1F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}
uint32_t compact3(uint64_t x) {
    x &= 0x1249249249249249ull;
    x = (x | (x >> 2)) & 0x10C30C30C30C30C3ull;
    x = (x | (x >> 4)) & 0x100F00F00F00F00Full;
    x = (x | (x >> 8)) & 0x1F0000FF0000FFull;
    x = (x | (x >> 16)) & 0x1F00000000FFFFull;
    x = (x | (x >> 32)) & 0x1FFFFF;
    return (uint32_t)x;
}
// Morton key: bits of i above those of j above those of k in every triple.
uint64_t morton(uint32_t i, uint32_t j, uint32_t k) { return (spread3(i) << 2) | (spread3(j) << 1) | spread3(k); }

int pass_chunk(int rp) {
    const int parts = (rp + 191) / 192;
    return ((rp + parts - 1) / parts + 15) / 16 * 16;
}

int ensure_pass_ops(kifmm_m2l_plan plan) {
    if (plan->pass_kept > 0) return KIFMM_OK;
    PassOps ops;
    int st = compute_pass_ops(plan->prm.p, plan->prm.d, plan->r, plan->U64, kPassRcond, ops);
    if (st != KIFMM_OK) return st;
    const size_t n = plan->n, r = plan->r, rp = plan->rp;
    // Ws in FP64 [rp][n]: output coefficient a, check point i (the per-point
    // S~ / T~ rows are formed from it on the device)
    {
        std::vector<double> w(rp * n, 0.0);
        for (size_t a = 0; a < r; ++a)
            for (size_t i = 0; i < n; ++i) w[a * n + i] = ops.Ws[a * n + i];
        KIFMM_CUDA_TRY(plan->Ws64.upload(w.data(), w.size()));
    }
    // M~_c as B [8][rp][rp] (B[a][b] = M~_c[a][b]) and L~_c = M~_c^T
    st = upload_pieces(plan->Mb, 8 * rp * rp, [&](size_t e) -> double {
        const size_t c = e / (rp * rp), a = (e / rp) % rp, b = e % rp;
        return (a < r && b < r) ? ops.Mt[(c * r + a) * r + b] : 0.0;
    });
    if (st != KIFMM_OK) return st;
    st = upload_pieces(plan->Lb, 8 * rp * rp, [&](size_t e) -> double {
        const size_t c = e / (rp * rp), a = (e / rp) % rp, b = e % rp;
        return (a < r && b < r) ? ops.Mt[(c * r + b) * r + a] : 0.0;
    });
    if (st != KIFMM_OK) return st;
    plan->pass_rcond = kPassRcond;
    plan->pass_kept = ops.kept;
    return KIFMM_OK;
}

}  // namespace

struct kifmm_fmm_s {
    kifmm_m2l_plan plan = nullptr;
    int instance = 0, depth = 0;
    double r0 = 0, centre[3] = {0, 0, 0};
    int64_t n_points = 0, n_pairs = 0, n_near = 0;
    std::vector<int> nbox;       // boxes per level, [depth + 1]
    std::vector<int64_t> off;    // first row of level l in the level-2..depth rows
    int64_t rows = 0;            // boxes of levels 2..depth
    struct Pass {
        int n_tiles = 0;
        int64_t tile0 = 0;       // first tile in the concatenated tables
    };
    std::vector<Pass> up, down;  // indexed by the parent level
    DevBuf<int> up_src, up_dst, up_k, dn_src, dn_dst, dn_k;
    DevBuf<float4> hi, lo;  // points in leaf units: hi (w = density) + lo
    DevBuf<float4> nhi, nlo;       // double layer: normals as two FP32 words (leaf order)
    bool dl = false;
    std::vector<int32_t> h_perm;   // caller's index of every leaf-ordered point
    DevBuf<int> perm, leaf_start, near_start, near_idx;
    DevBuf<int4> leaf_ijk;
    DevBuf<__nv_bfloat16> qb3, sl;
    DevBuf<float> qf, pt, qs;
    // per-point compressed rows [n_points][rp] (FP64-formed, stored FP32):
    // T~ rows (far field at a point; for point charges also their S~ rows)
    // and, with normals, the dipoles' S~ rows
    DevBuf<float> trows, drows;
    DevBuf<double> s64, xsurf64;  // points [n_points][3] and check points [n][3] in leaf units
    DevBuf<__nv_bfloat16> qh;
    int max_level_boxes = 0, max_down_tiles = 0;
};

namespace {

// GEMM over one level's M~ or L~ table: D[dst] += B_c A[src] (E_RED).
int pass_gemm(kifmm_m2l_plan plan, const __nv_bfloat16* A, long a_stride, int zero_row, const __nv_bfloat16* B,
              const int* src, const int* dst, const int* k, int n_tiles, float* D, cudaStream_t s) {
    if (n_tiles <= 0) return KIFMM_OK;
    UmmaArgs a{};
    a.A = A;
    a.a_piece_stride = a_stride;
    a.kdim = plan->rp;
    a.B = B;
    a.b_groups = 8;
    a.ndim = plan->rp;
    a.n_chunk = pass_chunk(plan->rp);
    a.row_src = src;
    a.row_dst = dst;
    a.tile_k = k;
    a.n_tiles = n_tiles;
    a.nrhs = 1;
    a.zero_row = zero_row;
    a.level_scale[0] = 1.0f;
    a.D = D;
    a.ldd = plan->rp;
    a.n_products = 6;
    a.hilo = 1;
    a.core_drain = 1;
    a.error_flag = plan->err_flag.ptr;
    KIFMM_CUDA_TRY(launch_umma(A_GATHER, E_RED, a, plan->num_sms, s));
    return KIFMM_OK;
}

// Children of parent level lp grouped by octant, 128 per tile: one row per
// child with src = src_of(child), dst = dst_of(child).
template <class SrcOf, class DstOf>
void octant_tables(const std::vector<int>& octant, SrcOf src_of, DstOf dst_of, std::vector<int32_t>& src,
                   std::vector<int32_t>& dst, std::vector<int32_t>& kk, int& n_tiles) {
    n_tiles = 0;
    for (int c = 0; c < 8; ++c) {
        std::vector<int> members;
        for (int e = 0; e < (int)octant.size(); ++e)
            if (octant[e] == c) members.push_back(e);
        for (size_t t0 = 0; t0 < members.size(); t0 += kTileRows) {
            for (int i = 0; i < kTileRows; ++i) {
                const size_t m = t0 + i;
                src.push_back(m < members.size() ? src_of(members[m]) : -1);
                dst.push_back(m < members.size() ? dst_of(members[m]) : -1);
            }
            kk.push_back(c);
            ++n_tiles;
        }
    }
}

int build_tree(kifmm_fmm f, const double* points, const double* centre, double r0) {
    kifmm_m2l_plan plan = f->plan;
    const int L = f->depth;
    const int64_t N = f->n_points;
    const uint32_t m = 1u << L;
    if (!(r0 > 0)) {
        double lo[3], hi[3];
        for (int t = 0; t < 3; ++t) lo[t] = hi[t] = points[t];
        for (int64_t i = 0; i < N; ++i)
            for (int t = 0; t < 3; ++t) {
                lo[t] = std::min(lo[t], points[3 * i + t]);
                hi[t] = std::max(hi[t], points[3 * i + t]);
            }
        double ext = 0;
        for (int t = 0; t < 3; ++t) {
            f->centre[t] = 0.5 * (lo[t] + hi[t]);
            ext = std::max(ext, 0.5 * (hi[t] - lo[t]));
        }
        f->r0 = ext * (1.0 + std::ldexp(1.0, -20));
        if (!(f->r0 > 0)) f->r0 = 1.0;  // all points coincide
    } else {
        for (int t = 0; t < 3; ++t) f->centre[t] = centre[t];
        f->r0 = r0;
    }
    // leaf of every point: floor((x - (c - r0)) / (2 r0) * 2^L), clamped
    std::vector<uint64_t> key(N);
    std::vector<uint32_t> ijk((size_t)3 * N);
    for (int64_t i = 0; i < N; ++i) {
        for (int t = 0; t < 3; ++t) {
            const double rel = (points[3 * i + t] - (f->centre[t] - f->r0)) / (2.0 * f->r0);
            double v = std::floor(rel * (double)m);
            v = std::min(std::max(v, 0.0), (double)(m - 1));
            ijk[3 * i + t] = (uint32_t)v;
        }
        key[i] = morton(ijk[3 * i], ijk[3 * i + 1], ijk[3 * i + 2]);
    }
    std::vector<int32_t> order(N);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
    // leaves and per-level boxes (Morton order at every level)
    std::vector<std::vector<uint64_t>> keys(L + 1);
    std::vector<int32_t> leaf_start;
    for (int64_t s = 0; s < N; ++s) {
        const uint64_t k = key[order[s]];
        if (keys[L].empty() || keys[L].back() != k) {
            keys[L].push_back(k);
            leaf_start.push_back((int32_t)s);
        }
    }
    leaf_start.push_back((int32_t)N);
    for (int l = L - 1; l >= 0; --l)
        for (uint64_t k : keys[l + 1])
            if (keys[l].empty() || keys[l].back() != (k >> 3)) keys[l].push_back(k >> 3);
    f->nbox.assign(L + 1, 0);
    for (int l = 0; l <= L; ++l) f->nbox[l] = (int)keys[l].size();
    auto box_ijk = [&](int l) {
        std::vector<int32_t> b((size_t)3 * keys[l].size());
        for (size_t e = 0; e < keys[l].size(); ++e) {
            b[3 * e] = (int32_t)compact3(keys[l][e] >> 2);
            b[3 * e + 1] = (int32_t)compact3(keys[l][e] >> 1);
            b[3 * e + 2] = (int32_t)compact3(keys[l][e]);
        }
        return b;
    };
    auto find = [&](int l, uint64_t k) -> int {
        auto it = std::lower_bound(keys[l].begin(), keys[l].end(), k);
        return (it != keys[l].end() && *it == k) ? (int)(it - keys[l].begin()) : -1;
    };
    // M2L levels 2..L on the plan, rows of the levels back to back
    f->off.assign(L + 1, -1);
    f->rows = 0;
    for (int l = 2; l <= L; ++l) {
        const std::vector<int32_t> b = box_ijk(l);
        int st = register_level(plan, f->instance, l, f->r0, f->nbox[l], b.data());
        if (st != KIFMM_OK) return st;
        f->off[l] = f->rows;
        f->rows += f->nbox[l];
        f->n_pairs += find_level(plan, f->instance, l)->n_pairs;
        f->max_level_boxes = std::max(f->max_level_boxes, f->nbox[l]);
    }
    MultiState* ms = nullptr;
    int st = get_multi_state(plan, f->instance, 2, L, false, &ms);
    if (st != KIFMM_OK) return st;
    TileSet* ts = nullptr;
    st = multi_tileset(*ms, 1, &ts);
    if (st != KIFMM_OK) return st;
    // M~ and L~ tables, by parent level
    f->up.assign(L + 1, {});
    f->down.assign(L + 1, {});
    std::vector<int32_t> us, ud, uk, ds, dd, dk;
    for (int lp = 2; lp < L; ++lp) {
        const int lc = lp + 1;
        std::vector<int> oct(f->nbox[lc]), par(f->nbox[lc]);
        for (int e = 0; e < f->nbox[lc]; ++e) {
            const uint64_t k = keys[lc][e];
            oct[e] = (int)(k & 7);  // low triple = (i & 1, j & 1, k & 1) = 4 b_x + 2 b_y + b_z
            par[e] = find(lp, k >> 3);
        }
        f->up[lp].tile0 = (int64_t)uk.size();
        octant_tables(
            oct, [&](int e) { return (int32_t)(f->off[lc] + e); }, [&](int e) { return (int32_t)par[e]; }, us, ud, uk,
            f->up[lp].n_tiles);
        f->down[lp].tile0 = (int64_t)dk.size();
        octant_tables(
            oct, [&](int e) { return (int32_t)par[e]; }, [&](int e) { return (int32_t)(f->off[lc] + e); }, ds, dd, dk,
            f->down[lp].n_tiles);
        f->max_down_tiles = std::max(f->max_down_tiles, (f->nbox[lp] + kTileRows - 1) / kTileRows);
    }
    KIFMM_CUDA_TRY(f->up_src.upload(us.data(), us.size()));
    KIFMM_CUDA_TRY(f->up_dst.upload(ud.data(), ud.size()));
    KIFMM_CUDA_TRY(f->up_k.upload(uk.data(), uk.size()));
    KIFMM_CUDA_TRY(f->dn_src.upload(ds.data(), ds.size()));
    KIFMM_CUDA_TRY(f->dn_dst.upload(dd.data(), dd.size()));
    KIFMM_CUDA_TRY(f->dn_k.upload(dk.data(), dk.size()));
    // leaves: coordinates, near lists
    const int B = f->nbox[L];
    const double h = f->r0 / (double)m;
    const std::vector<int32_t> lijk = box_ijk(L);
    std::vector<int4> h_lijk(B);
    std::vector<float4> h_hi(N), h_lo(N);
    std::vector<double> h_s64((size_t)N * 3);
    std::vector<int32_t> near_start(B + 1, 0), near_idx;
    for (int b = 0; b < B; ++b) {
        h_lijk[b] = make_int4(lijk[3 * b], lijk[3 * b + 1], lijk[3 * b + 2], 0);
        double c[3];
        for (int t = 0; t < 3; ++t) c[t] = (f->centre[t] - f->r0) + (2.0 * lijk[3 * b + t] + 1.0) * h;
        for (int s = leaf_start[b]; s < leaf_start[b + 1]; ++s) {
            const int64_t i = order[s];
            // leaf units s = (x - c) / h: hi on the 2^-20 grid (exact in FP32 for
            // |s| < 4, i.e. for every point inside the root cube), lo the rest
            float hv[3], lv[3];
            for (int t = 0; t < 3; ++t) {
                const double v = (points[3 * i + t] - c[t]) / h;
                h_s64[3 * (size_t)s + t] = v;
                hv[t] = (float)(std::nearbyint(v * 1048576.0) / 1048576.0);
                lv[t] = (float)(v - (double)hv[t]);
            }
            h_hi[s] = make_float4(hv[0], hv[1], hv[2], 0.f);
            h_lo[s] = make_float4(lv[0], lv[1], lv[2], 0.f);
        }
        const int64_t nt = leaf_start[b + 1] - leaf_start[b];
        // the leaf itself first, then its neighbours
        near_idx.push_back(b);
        f->n_near += nt * (nt - 1);
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dz = -1; dz <= 1; ++dz) {
                    const int64_t x = lijk[3 * b] + dx, y = lijk[3 * b + 1] + dy, z = lijk[3 * b + 2] + dz;
                    if (x < 0 || y < 0 || z < 0 || x >= m || y >= m || z >= m) continue;
                    const int s = find(L, morton((uint32_t)x, (uint32_t)y, (uint32_t)z));
                    if (s < 0 || s == b) continue;
                    near_idx.push_back(s);
                    f->n_near += nt * (leaf_start[s + 1] - leaf_start[s]);
                }
        near_start[b + 1] = (int32_t)near_idx.size();
    }
    KIFMM_CUDA_TRY(f->hi.upload(h_hi.data(), h_hi.size()));
    KIFMM_CUDA_TRY(f->lo.upload(h_lo.data(), h_lo.size()));
    KIFMM_CUDA_TRY(f->perm.upload(order.data(), order.size()));
    f->h_perm = order;
    KIFMM_CUDA_TRY(f->leaf_start.upload(leaf_start.data(), leaf_start.size()));
    KIFMM_CUDA_TRY(f->leaf_ijk.upload(h_lijk.data(), h_lijk.size()));
    KIFMM_CUDA_TRY(f->near_start.upload(near_start.data(), near_start.size()));
    KIFMM_CUDA_TRY(f->near_idx.upload(near_idx.data(), near_idx.size()));
    const std::vector<double> u = unit_surface(plan->prm.p);
    std::vector<double> h_x(3 * (size_t)plan->n);
    const double a_surf = 3.0 - 2.0 * plan->prm.d;  // upward check = downward equivalent surface, leaf units
    for (int i = 0; i < plan->n; ++i)
        for (int t = 0; t < 3; ++t) h_x[3 * i + t] = a_surf * u[3 * i + t];
    KIFMM_CUDA_TRY(f->xsurf64.upload(h_x.data(), h_x.size()));
    KIFMM_CUDA_TRY(f->s64.upload(h_s64.data(), h_s64.size()));
    // T~ rows of every point, in FP64: t(s)[a] = 1/(4 pi) sum_i Ws[a][i] / |x_i - s|
    // (leaf units).  For point charges the same row is the point's S~ row: the
    // upward check surface is the downward equivalent surface and G is symmetric.
    const size_t rp = plan->rp;
    KIFMM_CUDA_TRY(f->trows.ensure((size_t)N * rp));
    KIFMM_CUDA_TRY(launch_point_rows(f->s64.ptr, nullptr, (int)N, plan->Ws64.ptr, (int)rp, plan->n, f->xsurf64.ptr,
                                     0.0795774715459476679, f->trows.ptr, 0));
    KIFMM_CUDA_TRY(cudaStreamSynchronize(0));
    // scratch
    KIFMM_CUDA_TRY(f->qb3.ensure((size_t)3 * (f->rows + 1) * rp));
    KIFMM_CUDA_TRY(cudaMemset(f->qb3.ptr, 0, f->qb3.count * sizeof(__nv_bfloat16)));
    KIFMM_CUDA_TRY(f->pt.ensure((size_t)f->rows * rp));
    KIFMM_CUDA_TRY(f->qf.ensure((size_t)std::max<int64_t>(f->rows, 1) * rp));
    if (plan->prm.precision == KIFMM_PREC_F16X3) {
        KIFMM_CUDA_TRY(f->qh.ensure((size_t)2 * (f->rows + 1) * rp));
        KIFMM_CUDA_TRY(f->qs.ensure((size_t)f->rows + 1));
    }
    KIFMM_CUDA_TRY(f->sl.ensure((size_t)3 * (f->max_down_tiles + 1) * kTileRows * rp));
    return KIFMM_OK;
}

int evaluate(kifmm_fmm f, const float* q, float* out, int parts, cudaStream_t s) {
    kifmm_m2l_plan plan = f->plan;
    const int L = f->depth, B = f->nbox[L];
    const int rp = plan->rp;
    const double h = f->r0 / (double)(1u << L);
    const int N = (int)f->n_points;
    KIFMM_CUDA_TRY(launch_gather_density(q, f->perm.ptr, f->hi.ptr, N, s));
    const float4* nhi = f->dl ? f->nhi.ptr : nullptr;
    const float4* nlo = f->dl ? f->nlo.ptr : nullptr;
    if (parts & KIFMM_FMM_FAR) {
        const long qstride = (f->rows + 1) * rp;
        // S~ at the leaves through the per-point rows: q~_b = sum_{j in b} q_j s_j
        // (point charges: s_j is the point's T~ row; dipoles: its own S~ row),
        // into the leaf rows of qf and their BF16 pieces in qb3
        KIFMM_CUDA_TRY(launch_leaf_rows_sum(f->dl ? f->drows.ptr : f->trows.ptr, f->hi.ptr, f->leaf_start.ptr, B, rp,
                                            f->qf.ptr + f->off[L] * rp, f->qb3.ptr + f->off[L] * rp, qstride, s));
        // M~: q~_parent = sum_c M~_c q~_child, level by level towards the root
        for (int lp = L - 1; lp >= 2; --lp) {
            const auto& ps = f->up[lp];
            const int nb = f->nbox[lp];
            float* ql = f->qf.ptr + f->off[lp] * rp;
            KIFMM_CUDA_TRY(launch_zero(ql, (long)nb * rp, s));
            int st = pass_gemm(plan, f->qb3.ptr, qstride, (int)f->rows, plan->Mb.ptr, f->up_src.ptr + ps.tile0 * kTileRows,
                               f->up_dst.ptr + ps.tile0 * kTileRows, f->up_k.ptr + ps.tile0, ps.n_tiles, ql, s);
            if (st != KIFMM_OK) return st;
            KIFMM_CUDA_TRY(launch_split_rows(ql, nb, rp, rp, rp, nullptr, 0, (nb + kTileRows - 1) / kTileRows,
                                             f->qb3.ptr + f->off[lp] * rp, qstride, 3, s, /*pad_rows=*/0));
        }
        // M2L: p~ = s_l sum K~_o q~ over every level's pairs
        KIFMM_CUDA_TRY(launch_zero(f->pt.ptr, (long)f->rows * rp, s));
        {
            MultiState* ms = nullptr;
            int st = get_multi_state(plan, f->instance, 2, L, false, &ms);
            if (st != KIFMM_OK) return st;
            TileSet* ts = nullptr;
            st = multi_tileset(*ms, 1, &ts);
            if (st != KIFMM_OK) return st;
            ScaleTable scales{};
            for (int l = 2; l <= L; ++l) scales.s[l - 2] = (float)std::ldexp(1.0 / f->r0, l);
            if (plan->prm.precision == KIFMM_PREC_F16X3) {
                // the core's operand: every level's q~ as scaled FP16 pieces
                st = split_core_operand_f16(plan, f->qf.ptr, f->rows, f->qh.ptr, qstride, f->qs.ptr, s);
                if (st != KIFMM_OK) return st;
                st = launch_core(plan, f->qh.ptr, qstride, (int)f->rows, *ts, 1, scales, f->pt.ptr, s, f->qs.ptr);
            } else {
                st = launch_core(plan, f->qb3.ptr, qstride, (int)f->rows, *ts, 1, scales, f->pt.ptr, s);
            }
            if (st != KIFMM_OK) return st;
        }
        // L~: p~_child += L~_c p~_parent, level by level away from the root
        for (int lp = 2; lp < L; ++lp) {
            const auto& ps = f->down[lp];
            const int nb = f->nbox[lp], tiles = (nb + kTileRows - 1) / kTileRows;
            const long sstride = (long)(tiles + 1) * kTileRows * rp;
            KIFMM_CUDA_TRY(launch_split_rows(f->pt.ptr + f->off[lp] * rp, nb, rp, rp, rp, nullptr, 0, tiles + 1, f->sl.ptr,
                                             sstride, 3, s));
            int st = pass_gemm(plan, f->sl.ptr, sstride, tiles * kTileRows, plan->Lb.ptr,
                               f->dn_src.ptr + ps.tile0 * kTileRows, f->dn_dst.ptr + ps.tile0 * kTileRows,
                               f->dn_k.ptr + ps.tile0, ps.n_tiles, f->pt.ptr, s);
            if (st != KIFMM_OK) return st;
        }
    }
    // leaf sums: the far field as T~ row . p~_leaf (T~ and L2T of Sec. 3.3 in one
    // r-long dot product per point) plus the near field, in the caller's order
    KIFMM_CUDA_TRY(launch_leaf_eval(f->hi.ptr, f->lo.ptr, nhi, nlo, f->leaf_start.ptr, f->leaf_ijk.ptr, f->near_start.ptr,
                                    f->near_idx.ptr, B, f->trows.ptr, rp, f->pt.ptr + f->off[L] * rp,
                                    (float)(0.0795774715459476679 / h), (float)(0.0795774715459476679 / (h * h)),
                                    f->perm.ptr, out, parts, s));
    return KIFMM_OK;
}

void drop_levels(kifmm_fmm f) {
    kifmm_m2l_plan plan = f->plan;
    if (!plan) return;
    plan->fmms.erase(f);
    for (auto it = plan->levels.begin(); it != plan->levels.end();)
        it = it->first.first == f->instance ? plan->levels.erase(it) : std::next(it);
    for (auto it = plan->multi.begin(); it != plan->multi.end();)
        it = std::get<0>(it->first) == f->instance ? plan->multi.erase(it) : std::next(it);
}

}  // namespace

namespace kifmm {

void detach_fmms(kifmm_m2l_plan plan) {
    for (kifmm_fmm f : plan->fmms) f->plan = nullptr;
    plan->fmms.clear();
}

}  // namespace kifmm

extern "C" {

int kifmm_fmm_create(kifmm_m2l_plan plan, int64_t n_points, const double* points, int depth, const double* centre,
                     double r0, kifmm_fmm* out) {
    if (!out) {
        set_error("out is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!plan || !points) {
        set_error("plan or points is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (n_points < 1 || n_points >= (int64_t)1 << 30) {
        set_error("need 1 <= n_points < 2^30");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (depth < 2 || depth > 20) {
        set_error("need 2 <= depth <= 20");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (r0 > 0 && (!centre || !std::isfinite(r0) || !std::isfinite(centre[0]) || !std::isfinite(centre[1]) ||
                   !std::isfinite(centre[2]))) {
        set_error("r0 > 0 needs a finite centre and r0");
        return KIFMM_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < 3 * n_points; ++i)
        if (!std::isfinite(points[i])) {
            set_error("non-finite point coordinate at index " + std::to_string(i / 3));
            return KIFMM_ERR_INVALID_ARG;
        }
    if (plan->prm.precision == KIFMM_PREC_FP32) {
        set_error("point-source evaluation runs its passes on the tensor cores: use a BF16 / split / f16x3 precision");
        return KIFMM_ERR_UNSUPPORTED;
    }
    if (plan->prm.kernel_id != KIFMM_KERNEL_LAPLACE) {
        set_error("point-source evaluation is built for the Laplace kernel");
        return KIFMM_ERR_UNSUPPORTED;
    }
    if (plan->n > 512) {
        set_error("point-source evaluation supports n <= 512 surface points (p <= 10)");
        return KIFMM_ERR_UNSUPPORTED;
    }
    int st = check_device(plan);
    if (st != KIFMM_OK) return st;
    std::unique_ptr<kifmm_fmm_s> f;
    try {
        st = ensure_pass_ops(plan);
        if (st != KIFMM_OK) return st;
        f.reset(new kifmm_fmm_s());
        f->plan = plan;
        f->depth = depth;
        f->n_points = n_points;
        f->instance = kReservedInstance + plan->next_fmm_instance++;
        plan->fmms.insert(f.get());
        st = build_tree(f.get(), points, centre, r0);
        if (st != KIFMM_OK) {
            drop_levels(f.get());
            return st;
        }
    } catch (const std::bad_alloc&) {
        if (f) drop_levels(f.get());
        set_error("host allocation failed");
        return KIFMM_ERR_OOM;
    }
    *out = f.release();
    return KIFMM_OK;
}

int kifmm_fmm_evaluate(kifmm_fmm fmm, const float* q, float* potential, int parts, void* stream) {
    if (!fmm || !q || !potential) {
        set_error("fmm, q or potential is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (parts < 1 || parts > 3) {
        set_error("parts must be KIFMM_FMM_NEAR, KIFMM_FMM_FAR or both");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (!fmm->plan) {
        set_error("the plan of this tree was destroyed");
        return KIFMM_ERR_STATE;
    }
    int st = check_device(fmm->plan);
    if (st != KIFMM_OK) return st;
    return evaluate(fmm, q, potential, parts, static_cast<cudaStream_t>(stream));
}

int kifmm_fmm_set_normals(kifmm_fmm fmm, const double* normals) {
    if (!fmm) {
        set_error("fmm is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (!normals) {
        fmm->dl = false;
        return KIFMM_OK;
    }
    const int64_t N = fmm->n_points;
    for (int64_t i = 0; i < 3 * N; ++i)
        if (!std::isfinite(normals[i])) {
            set_error("non-finite normal at index " + std::to_string(i / 3));
            return KIFMM_ERR_INVALID_ARG;
        }
    if (fmm->plan) {
        int st = check_device(fmm->plan);
        if (st != KIFMM_OK) return st;
    }
    try {
        std::vector<float4> vh((size_t)N), vl((size_t)N);
        std::vector<double> v64((size_t)N * 3);
        for (int64_t s = 0; s < N; ++s) {
            const double* v = normals + 3 * (int64_t)fmm->h_perm[s];
            float w[3], r[3];
            for (int t = 0; t < 3; ++t) {
                w[t] = (float)v[t];
                r[t] = (float)(v[t] - (double)w[t]);
                v64[3 * s + t] = v[t];
            }
            vh[s] = make_float4(w[0], w[1], w[2], 0.f);
            vl[s] = make_float4(r[0], r[1], r[2], 0.f);
        }
        KIFMM_CUDA_TRY(fmm->nhi.upload(vh.data(), vh.size()));
        KIFMM_CUDA_TRY(fmm->nlo.upload(vl.data(), vl.size()));
        if (fmm->plan) {
            // the dipoles' S~ rows in FP64: s(y)[a] = 1/(4 pi h) sum_i Ws[a][i]
            // n . (x_i - y) / |x_i - y|^3 (leaf units; the first step of S2M for a
            // double layer, Eq. (26))
            kifmm_m2l_plan plan = fmm->plan;
            const double h = fmm->r0 / (double)(1u << fmm->depth);
            DevBuf<double> n64;
            KIFMM_CUDA_TRY(n64.upload(v64.data(), v64.size()));
            KIFMM_CUDA_TRY(fmm->drows.ensure((size_t)N * plan->rp));
            KIFMM_CUDA_TRY(launch_point_rows(fmm->s64.ptr, n64.ptr, (int)N, plan->Ws64.ptr, plan->rp, plan->n,
                                             fmm->xsurf64.ptr, 0.0795774715459476679 / h, fmm->drows.ptr, 0));
            KIFMM_CUDA_TRY(cudaStreamSynchronize(0));
        }
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return KIFMM_ERR_OOM;
    }
    fmm->dl = true;
    return KIFMM_OK;
}

int kifmm_fmm_info(kifmm_fmm fmm, int* depth, int64_t* n_leaves, int64_t* n_boxes, int64_t* n_m2l_pairs,
                   int64_t* n_near_pairs) {
    if (!fmm) {
        set_error("fmm is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (depth) *depth = fmm->depth;
    if (n_leaves) *n_leaves = fmm->nbox[fmm->depth];
    if (n_boxes) *n_boxes = fmm->rows;
    if (n_m2l_pairs) *n_m2l_pairs = fmm->n_pairs;
    if (n_near_pairs) *n_near_pairs = fmm->n_near;
    return KIFMM_OK;
}

int kifmm_fmm_destroy(kifmm_fmm fmm) {
    if (!fmm) return KIFMM_OK;
    drop_levels(fmm);
    delete fmm;
    return KIFMM_OK;
}

int kifmm_m2l_pass_ops_host(const kifmm_m2l_params* params, double rcond, int* kept, double* Ws, double* Mt) {
    if (params && params->kernel_id != KIFMM_KERNEL_LAPLACE) {
        set_error("the pass operators are built for the Laplace kernel");
        return KIFMM_ERR_UNSUPPORTED;
    }
    Factors f;
    int st = compute_factors(*params, f);
    if (st != KIFMM_OK) return st;
    PassOps ops;
    st = compute_pass_ops(params->p, params->d, f.r, f.U, rcond, ops);
    if (st != KIFMM_OK) return st;
    if (kept) *kept = ops.kept;
    if (Ws) std::copy(ops.Ws.begin(), ops.Ws.end(), Ws);
    if (Mt) std::copy(ops.Mt.begin(), ops.Mt.end(), Mt);
    return KIFMM_OK;
}

}  // extern "C"
