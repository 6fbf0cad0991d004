// Host-side set-up of a context's layouts: CSR validation, the per-diagonal
// (stencil) and CSR layouts with the reverse-edge index and the edge
// coefficients, the reverse Cuthill-McKee renumbering, and the line and
// parity-class schedules' data.
#include "host.h"

namespace gabp {

// ---------------------------------------------------------------------------
// CSR validation and layout construction (host)
// ---------------------------------------------------------------------------
gabp_status validate_csr(int32_t n, int64_t nnz, const int64_t *indptr, const int32_t *indices,
                         const double *data)
{
    if (n < 0 || nnz < 0) return fail(GABP_E_INVALID_ARG, "negative size");
    if (n > 0 && (!indptr || (nnz > 0 && (!indices || !data))))
        return fail(GABP_E_INVALID_ARG, "null matrix array");
    if (n == 0) return GABP_OK;
    if (indptr[0] != 0 || indptr[n] != nnz) return fail(GABP_E_BAD_CSR, "indptr[0] != 0 or indptr[n] != nnz");
    for (int32_t r = 0; r < n; ++r) {
        if (indptr[r + 1] < indptr[r]) return fail(GABP_E_BAD_CSR, "indptr not monotone");
        bool diag = false;
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p) {
            const int32_t c = indices[p];
            if (c < 0 || c >= n) return fail(GABP_E_BAD_CSR, "column index out of range");
            if (p > indptr[r] && indices[p - 1] >= c)
                return fail(GABP_E_BAD_CSR, "columns not strictly ascending (unsorted or duplicate)");
            if (!std::isfinite(data[p])) return fail(GABP_E_BAD_CSR, "non-finite matrix value");
            if (c == r) {
                if (data[p] == 0.0) return fail(GABP_E_ZERO_DIAG, "zero diagonal entry in row " + std::to_string(r));
                diag = true;
            }
        }
        if (!diag) return fail(GABP_E_ZERO_DIAG, "missing diagonal entry in row " + std::to_string(r));
    }
    return GABP_OK;
}

// Distinct off-diagonal offsets closed under negation; false if more than KMAX.
bool stencil_offsets(int32_t n, const int64_t *indptr, const int32_t *indices, StencilParams &sp)
{
    std::vector<int> absoff;
    for (int32_t r = 0; r < n; ++r)
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p) {
            const int o = indices[p] - r;
            if (o == 0) continue;
            const int ao = o < 0 ? -o : o;
            if (std::find(absoff.begin(), absoff.end(), ao) == absoff.end()) {
                absoff.push_back(ao);
                if ((int)absoff.size() * 2 > KMAX) return false;
            }
        }
    std::sort(absoff.begin(), absoff.end());
    const int h = (int)absoff.size();
    sp.K = 2 * h;
    for (int i = 0; i < h; ++i) {
        sp.off[i] = -absoff[h - 1 - i];
        sp.off[h + i] = absoff[i];
    }
    for (int k = 0; k < sp.K; ++k) sp.krev[k] = sp.K - 1 - k;  // off sorted symmetric
    for (int k = sp.K; k < KMAX; ++k) sp.off[k] = sp.krev[k] = 0;
    return true;
}

void build_stencil(int32_t n, const int64_t *indptr, const int32_t *indices, const double *data,
                   const StencilParams &sp, HostLayout &H)
{
    H.kind = GABP_LAYOUT_STENCIL;
    H.sp = sp;
    const int K = sp.K;
    H.slots = (int64_t)K * n;
    H.a.assign((size_t)H.slots, 0.0);
    H.c.assign((size_t)H.slots, 0.0);
    H.diag.assign((size_t)n, 0.0);
    H.slotmap.assign((size_t)indptr[n], -1);
    for (int32_t r = 0; r < n; ++r) {
        int k = 0;
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p) {
            const int o = indices[p] - r;
            if (o == 0) {
                H.diag[r] = data[p];
                continue;
            }
            while (sp.off[k] != o) ++k;  // columns ascend, offsets ascend
            const int64_t e = (int64_t)k * n + r;
            H.a[e] = -data[p];
            H.slotmap[p] = e;
        }
    }
    for (int k = 0; k < K; ++k) {
        const int o = sp.off[k];
        const int64_t kr = sp.krev[k];
        for (int32_t r = 0; r < n; ++r) {
            const int64_t e = (int64_t)k * n + r;
            const int64_t s = (int64_t)r + o;
            if (H.a[e] != 0.0 && s >= 0 && s < n) H.c[e] = -H.a[e] * H.a[kr * n + s];
        }
    }
}

void build_csr(int32_t n, const int64_t *indptr, const int32_t *indices, const double *data,
               HostLayout &H)
{
    H.kind = GABP_LAYOUT_CSR;
    // symmetrised off-diagonal pattern
    std::vector<int64_t> cnt((size_t)n + 1, 0);
    for (int32_t r = 0; r < n; ++r)
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p)
            if (indices[p] != r) {
                cnt[r + 1]++;
                cnt[indices[p] + 1]++;
            }
    for (int32_t r = 0; r < n; ++r) cnt[r + 1] += cnt[r];
    std::vector<int> tmp((size_t)cnt[n]);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int32_t r = 0; r < n; ++r)
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p)
            if (indices[p] != r) {
                tmp[fill[r]++] = indices[p];
                tmp[fill[indices[p]]++] = r;
            }
    H.rowptr.assign((size_t)n + 1, 0);
    H.col.clear();
    H.col.reserve(tmp.size());
    for (int32_t r = 0; r < n; ++r) {
        auto b0 = tmp.begin() + cnt[r], b1 = tmp.begin() + cnt[r + 1];
        std::sort(b0, b1);
        auto e = std::unique(b0, b1);
        for (auto it = b0; it != e; ++it) H.col.push_back(*it);
        H.rowptr[r + 1] = (int)H.col.size();
    }
    H.slots = (int64_t)H.col.size();
    auto find = [&](int r, int s) -> int64_t {
        auto b0 = H.col.begin() + H.rowptr[r], b1 = H.col.begin() + H.rowptr[r + 1];
        auto it = std::lower_bound(b0, b1, s);
        return (it != b1 && *it == s) ? (int64_t)(it - H.col.begin()) : -1;
    };
    H.a.assign((size_t)H.slots, 0.0);
    H.c.assign((size_t)H.slots, 0.0);
    H.rev.assign((size_t)H.slots, 0);
    H.diag.assign((size_t)n, 0.0);
    H.slotmap.assign((size_t)indptr[n], -1);
    for (int32_t r = 0; r < n; ++r)
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p) {
            if (indices[p] == r) {
                H.diag[r] = data[p];
                continue;
            }
            const int64_t e = find(r, indices[p]);
            H.a[e] = -data[p];
            H.slotmap[p] = e;
        }
    for (int32_t r = 0; r < n; ++r)
        for (int e = H.rowptr[r]; e < H.rowptr[r + 1]; ++e) {
            const int64_t q = find(H.col[e], r);
            H.rev[e] = (int)q;
            H.c[e] = -H.a[e] * H.a[q];
        }
}

template <typename T>
std::vector<T> cast_vec(const std::vector<double> &v)
{
    std::vector<T> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = (T)v[i];
    return o;
}


// Uploads the coefficient arrays (a, c, diag in both precisions) of H.
gabp_status upload_coeffs(gabp_ctx *ctx, const HostLayout &H, bool realloc)
{
    const size_t S = (size_t)H.slots, n = (size_t)ctx->n;
    auto put = [&](void **dst, const void *src, size_t bytes) -> gabp_status {
        if (realloc) return upload(ctx, dst, src, bytes);
        if (bytes) CK(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
        return GABP_OK;
    };
    CKS(put((void **)&ctx->a64, H.a.data(), S * sizeof(double)));
    CKS(put((void **)&ctx->diag64, H.diag.data(), n * sizeof(double)));
    if (ctx->prec == 0) {
        ctx->a = ctx->a64;
        ctx->diagT = ctx->diag64;
        CKS(put(&ctx->c, H.c.data(), S * sizeof(double)));
    } else {
        auto af = cast_vec<float>(H.a), cf = cast_vec<float>(H.c), df = cast_vec<float>(H.diag);
        CKS(put(&ctx->a, af.data(), S * sizeof(float)));
        CKS(put(&ctx->c, cf.data(), S * sizeof(float)));
        CKS(put(&ctx->diagT, df.data(), n * sizeof(float)));
    }
    return GABP_OK;
}

// Symmetrised adjacency of A without the diagonal, rows sorted, no duplicates.
void sym_adjacency(int32_t n, const int64_t *indptr, const int32_t *indices,
                   std::vector<int64_t> &ap, std::vector<int32_t> &aj)
{
    std::vector<int64_t> cnt((size_t)n + 1, 0);
    for (int32_t r = 0; r < n; ++r)
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p)
            if (indices[p] != r) {
                cnt[r + 1]++;
                cnt[indices[p] + 1]++;
            }
    for (int32_t r = 0; r < n; ++r) cnt[r + 1] += cnt[r];
    std::vector<int32_t> tmp((size_t)cnt[n]);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int32_t r = 0; r < n; ++r)
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p)
            if (indices[p] != r) {
                tmp[fill[r]++] = indices[p];
                tmp[fill[indices[p]]++] = r;
            }
    ap.assign((size_t)n + 1, 0);
    aj.clear();
    aj.reserve(tmp.size());
    for (int32_t r = 0; r < n; ++r) {
        auto b0 = tmp.begin() + cnt[r], b1 = tmp.begin() + cnt[r + 1];
        std::sort(b0, b1);
        auto e = std::unique(b0, b1);
        aj.insert(aj.end(), b0, e);
        ap[r + 1] = (int64_t)aj.size();
    }
}

// Reverse Cuthill-McKee order of the symmetrised graph: for each connected
// component a breadth-first search from a pseudo-peripheral node (the last
// node a search from a minimum-degree node reaches), each node's unvisited
// neighbours taken by ascending degree; the whole order reversed.  perm[i] is
// the node placed at position i.  Returns whether the renumbering is worth it
// (`force`, or it at least halves the mean |i - j| over the coupled pairs).
bool rcm_order(int32_t n, const int64_t *indptr, const int32_t *indices, bool force,
               std::vector<int32_t> &perm)
{
    std::vector<int64_t> ap;
    std::vector<int32_t> aj;
    sym_adjacency(n, indptr, indices, ap, aj);
    auto deg = [&](int32_t v) { return ap[v + 1] - ap[v]; };
    std::vector<int32_t> byDeg((size_t)n);
    for (int32_t i = 0; i < n; ++i) byDeg[i] = i;
    std::stable_sort(byDeg.begin(), byDeg.end(), [&](int32_t a, int32_t b) { return deg(a) < deg(b); });
    std::vector<int32_t> stamp((size_t)n, -1);
    std::vector<char> placed((size_t)n, 0);
    std::vector<int32_t> order, queue, nb;
    order.reserve(n);
    queue.reserve(n);
    int32_t comp = 0;
    for (int32_t v0 : byDeg) {
        if (placed[v0]) continue;
        // pseudo-peripheral start: the last node reached from v0
        queue.clear();
        queue.push_back(v0);
        stamp[v0] = comp;
        for (size_t h = 0; h < queue.size(); ++h)
            for (int64_t p = ap[queue[h]]; p < ap[queue[h] + 1]; ++p)
                if (stamp[aj[p]] != comp) {
                    stamp[aj[p]] = comp;
                    queue.push_back(aj[p]);
                }
        const int32_t u = queue.back();
        // Cuthill-McKee from u
        const size_t first = order.size();
        order.push_back(u);
        placed[u] = 1;
        for (size_t h = first; h < order.size(); ++h) {
            const int32_t w = order[h];
            nb.clear();
            for (int64_t p = ap[w]; p < ap[w + 1]; ++p)
                if (!placed[aj[p]]) {
                    placed[aj[p]] = 1;
                    nb.push_back(aj[p]);
                }
            std::stable_sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) { return deg(a) < deg(b); });
            order.insert(order.end(), nb.begin(), nb.end());
        }
        ++comp;
    }
    std::reverse(order.begin(), order.end());
    perm.swap(order);
    if (force) return true;
    std::vector<int32_t> iperm((size_t)n);
    for (int32_t i = 0; i < n; ++i) iperm[perm[i]] = i;
    double before = 0.0, after = 0.0;
    for (int32_t r = 0; r < n; ++r)
        for (int64_t p = ap[r]; p < ap[r + 1]; ++p) {
            before += std::abs((double)aj[p] - r);
            after += std::abs((double)iperm[aj[p]] - iperm[r]);
        }
    return after * 2.0 <= before;
}

// The CSR of P A P^T for the order perm (internal row i = caller row perm[i]),
// rows sorted, and pmap[p] = position of the caller's entry p in it.
void permute_csr(int32_t n, const int64_t *indptr, const int32_t *indices,
                 const std::vector<int32_t> &perm, std::vector<int64_t> &pindptr,
                 std::vector<int32_t> &pindices, std::vector<int64_t> &pmap)
{
    std::vector<int32_t> iperm((size_t)n);
    for (int32_t i = 0; i < n; ++i) iperm[perm[i]] = i;
    pindptr.assign((size_t)n + 1, 0);
    for (int32_t i = 0; i < n; ++i) pindptr[i + 1] = pindptr[i] + (indptr[perm[i] + 1] - indptr[perm[i]]);
    pindices.assign((size_t)indptr[n], 0);
    pmap.assign((size_t)indptr[n], 0);
    std::vector<std::pair<int32_t, int64_t>> row;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t r = perm[i];
        row.clear();
        for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p) row.emplace_back(iperm[indices[p]], p);
        std::sort(row.begin(), row.end());
        int64_t q = pindptr[i];
        for (auto &cp : row) {
            pindices[q] = cp.first;
            pmap[cp.second] = q;
            ++q;
        }
    }
}

std::vector<double> permute_values(const std::vector<int64_t> &pmap, const double *data)
{
    std::vector<double> v(pmap.size());
    for (size_t p = 0; p < pmap.size(); ++p) v[pmap[p]] = data[p];
    return v;
}

gabp_status setup_lines(gabp_ctx *ctx)
{
    if (ctx->reordered)
        return fail(GABP_E_INVALID_ARG, "the line schedule needs the caller's grid numbering (reorder = 0)");
    const int n = ctx->n;
    int m = 0;
    while ((int64_t)m * m < n) ++m;
    if ((int64_t)m * m != n || n == 0) return fail(GABP_E_INVALID_ARG, "line schedule needs an m x m grid");
    const int64_t *ip = ctx->h_indptr.data();
    const int32_t *ix = ctx->h_indices.data();
    const double *dv = ctx->h_data.data();
    std::vector<double> subH(n, 0.0), supH(n, 0.0), subV(n, 0.0), supV(n, 0.0), dT(n, 0.0);
    std::vector<double> dg(n, 0.0);
    for (int r = 0; r < n; ++r) {
        const int rx = r % m, ry = r / m;
        for (int64_t p = ip[r]; p < ip[r + 1]; ++p) {
            const int j = ix[p];
            const int jx = j % m, jy = j / m;
            if (j == r) dg[r] = dv[p];
            else if (jy == ry && jx == rx - 1) subH[r] = dv[p];                      // west, along the row
            else if (jy == ry && jx == rx + 1) supH[r] = dv[p];                      // east
            else if (jx == rx && jy == ry - 1) subV[(size_t)rx * m + ry] = dv[p];   // south, along the column
            else if (jx == rx && jy == ry + 1) supV[(size_t)rx * m + ry] = dv[p];   // north
            else return fail(GABP_E_INVALID_ARG, "line schedule needs a 5-point grid matrix (every edge inside a row or a column)");
        }
    }
    for (int r = 0; r < n; ++r) dT[(size_t)(r % m) * m + r / m] = dg[r];
    const size_t nb = (size_t)n * esz(ctx->prec);
    auto put = [&](void **dst, const std::vector<double> &v) -> gabp_status {
        if (!*dst) CKS(dalloc(ctx, dst, nb));
        if (ctx->prec == 0) {
            CK(cudaMemcpy(*dst, v.data(), nb, cudaMemcpyHostToDevice));
        } else {
            auto f = cast_vec<float>(v);
            CK(cudaMemcpy(*dst, f.data(), nb, cudaMemcpyHostToDevice));
        }
        return GABP_OK;
    };
    CKS(put(&ctx->lsubH, subH));
    CKS(put(&ctx->lsupH, supH));
    CKS(put(&ctx->lsubV, subV));
    CKS(put(&ctx->lsupV, supV));
    CKS(put(&ctx->ldiagT, dT));
    void **bufs[] = {&ctx->lbT, &ctx->LH, &ctx->MH, &ctx->LV, &ctx->MV, &ctx->LHt, &ctx->MHt,
                     &ctx->LVt, &ctx->MVt};
    for (void **bp : bufs) {
        if (!*bp) CKS(dalloc(ctx, bp, nb));
        CK(cudaMemset(*bp, 0, nb));
    }
    if (line_needs_scratch(ctx->prec, m)) {
        if (!ctx->lf) CKS(dalloc(ctx, &ctx->lf, nb));
        if (!ctx->ly) CKS(dalloc(ctx, &ctx->ly, nb));
    }
    CK(prepare_line_kernels(ctx->prec, m));
    ctx->lines_m = m;
    return GABP_OK;
}

// Coloured schedule on the parity-class layout when A is an m x m grid
// stencil (m >= 3, every coupling inside the 3 x 3 neighbourhood, none
// wrapping around a grid row) and every colour is a union of parity classes.
// Leaves ctx->parity false when A or the colouring does not fit.
gabp_status setup_parity(gabp_ctx *ctx, const std::vector<int> &col, int nc)
{
    ctx->parity = false;
    const int n = ctx->n;
    const StencilParams &sp = ctx->L.sp;
    if (ctx->L.kind != GABP_LAYOUT_STENCIL || sp.K == 0 || sp.K > KMAXPG) return GABP_OK;
    int m = 0;
    while ((int64_t)m * m < n) ++m;
    if ((int64_t)m * m != n || m < 3) return GABP_OK;
    ParityGrid g{};
    g.m = m;
    g.K = sp.K;
    for (int k = 0; k < sp.K; ++k) {
        bool found = false;
        for (int dy = -1; dy <= 1 && !found; ++dy)
            for (int dx = -1; dx <= 1 && !found; ++dx)
                if ((dx || dy) && dy * m + dx == sp.off[k]) {
                    g.dx[k] = dx;
                    g.dy[k] = dy;
                    found = true;
                }
        if (!found) return GABP_OK;
        g.krev[k] = sp.krev[k];
    }
    const int64_t *ip = ctx->h_indptr.data();
    const int32_t *ix = ctx->h_indices.data();
    for (int r = 0; r < n; ++r)
        for (int64_t p = ip[r]; p < ip[r + 1]; ++p) {
            const int j = ix[p];
            if (j == r) continue;
            const int ddx = j % m - r % m, ddy = j / m - r / m;
            if (ddx < -1 || ddx > 1 || ddy < -1 || ddy > 1) return GABP_OK;
        }
    int qc[4] = {-1, -1, -1, -1};
    for (int i = 0; i < n; ++i) {
        const int q = ((i % m) & 1) | (((i / m) & 1) << 1);
        if (qc[q] < 0) qc[q] = col[i];
        else if (qc[q] != col[i]) return GABP_OK;
    }
    long long size[4], acc = 0;
    for (int q = 0; q < 4; ++q) {
        g.w[q] = (m - (q & 1) + 1) / 2;
        g.h[q] = (m - (q >> 1) + 1) / 2;
        size[q] = (long long)g.w[q] * g.h[q];
        g.base[q] = acc;
        acc += size[q];
    }
    // the full 3 x 3 neighbourhood (or its 5-point part) in ascending order
    static const int dx4[4] = {0, -1, 1, 0}, dy4[4] = {-1, 0, 0, 1};
    static const int dx8[8] = {-1, 0, 1, -1, 1, -1, 0, 1}, dy8[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
    g.std_order = (g.K == 4 || g.K == 8) && (long long)g.K * n < (1LL << 31);
    for (int k = 0; k < g.K && g.std_order; ++k) {
        const int ex = g.K == 4 ? dx4[k] : dx8[k], ey = g.K == 4 ? dy4[k] : dy8[k];
        if (g.dx[k] != ex || g.dy[k] != ey || g.krev[k] != g.K - 1 - k) g.std_order = 0;
    }
    std::vector<PhaseClasses> phases((size_t)nc);
    for (int c = 0; c < nc; ++c) {
        PhaseClasses &ph = phases[(size_t)c];
        ph = PhaseClasses{};
        for (int q = 0; q < 4; ++q)
            if (qc[q] == c) {
                ph.q[ph.nq] = q;
                ph.start[ph.nq + 1] = ph.start[ph.nq] + size[q];
                ++ph.nq;
            }
    }
    const size_t S = (size_t)ctx->L.slots * esz(ctx->prec);
    if (!ctx->pa) CKS(dalloc(ctx, &ctx->pa, S));
    if (!ctx->pc) CKS(dalloc(ctx, &ctx->pc, S));
    CK(launch_parity_convert(g, ctx->prec, 1, ctx->a, ctx->pa, ctx->stream));
    CK(launch_parity_convert(g, ctx->prec, 1, ctx->c, ctx->pc, ctx->stream));
    ctx->pg = g;
    ctx->phases.swap(phases);
    ctx->parity = true;
    if (ctx->aT) CKS(ensure_parity_transpose(ctx));
    return GABP_OK;
}

}  // namespace gabp
