// Theta-independent model set-up on the host (Sections II-A.1, II-A.2):
// P1 finite elements on the mesh, G C^{-1} G, barycentric interpolation of the
// observations, the observation Gram matrices per (time step, variable) and
// A^T y.  Everything that depends on theta is done on the device by the
// assembly kernels; this file runs once per model.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "common.cuh"

namespace {

struct Csr {
    std::vector<int> rowptr, col;
    std::vector<double> val;
};

// Row-wise accumulation into sorted maps, then CSR.
Csr to_csr(int n, const std::vector<std::map<int, double>>& rows) {
    Csr c;
    c.rowptr.resize(n + 1, 0);
    for (int i = 0; i < n; ++i) c.rowptr[i + 1] = c.rowptr[i] + (int)rows[i].size();
    c.col.reserve(c.rowptr[n]);
    c.val.reserve(c.rowptr[n]);
    for (int i = 0; i < n; ++i)
        for (const auto& kv : rows[i]) {
            c.col.push_back(kv.first);
            c.val.push_back(kv.second);
        }
    return c;
}

// Position of column j in row i of a CSR pattern (binary search), -1 if absent.
int find_pos(const std::vector<int>& rowptr, const std::vector<int>& col, int i, int j) {
    auto b = col.begin() + rowptr[i], e = col.begin() + rowptr[i + 1];
    auto it = std::lower_bound(b, e, j);
    return (it != e && *it == j) ? (int)(it - col.begin()) : -1;
}

template <class T>
int upload(T** dst, const std::vector<T>& src) {
    size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
    cudaError_t e = cudaMalloc((void**)dst, bytes);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? BTA_ERR_OOM : bta_cuda_fail(e);
    if (!src.empty()) BTA_CUDA_TRY(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T),
                                              cudaMemcpyHostToDevice));
    return BTA_OK;
}

}  // namespace

extern "C" int bta_model_create(const bta_model_desc* d, bta_model_t* out) {
    if (!d || !out) return BTA_ERR_ARG;
    *out = nullptr;
    const int nv = d->nv, ns = d->ns, nt = d->nt, nr = d->nr, m = d->m;
    if (nv < 1 || nv > BTA_MAX_NV || ns < 3 || nt < 1 || nr < 0 || m < 0 || d->n_tri < 1)
        return BTA_ERR_ARG;
    if (!d->nodes || !d->tri || (m > 0 && (!d->obs_var || !d->obs_time || !d->obs_xy ||
                                           !d->obs_tri || !d->y || (nr > 0 && !d->X))))
        return BTA_ERR_ARG;
    const int dim_theta = 4 * nv + nv * (nv - 1) / 2;
    const int b = nv * ns, a = nv * nr, n = nt;
    const long long N = (long long)n * b + a;

    // --- P1 elements: lumped mass and stiffness -----------------------------------------
    std::vector<double> C(ns, 0.0);
    std::vector<std::map<int, double>> Grows(ns);
    for (int t = 0; t < d->n_tri; ++t) {
        int v[3];
        for (int q = 0; q < 3; ++q) {
            v[q] = d->tri[3 * t + q];
            if (v[q] < 0 || v[q] >= ns) return BTA_ERR_ARG;
        }
        double x[3], y[3];
        for (int q = 0; q < 3; ++q) {
            x[q] = d->nodes[2 * v[q]];
            y[q] = d->nodes[2 * v[q] + 1];
        }
        // twice the signed area
        double det = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
        double area = 0.5 * std::fabs(det);
        if (!(area > 0)) return BTA_ERR_ARG;
        // gradient of the hat function of vertex q: rotate the opposite edge
        double gx[3], gy[3];
        for (int q = 0; q < 3; ++q) {
            int q1 = (q + 1) % 3, q2 = (q + 2) % 3;
            gx[q] = (y[q1] - y[q2]) / det;
            gy[q] = (x[q2] - x[q1]) / det;
        }
        for (int q = 0; q < 3; ++q) {
            C[v[q]] += area / 3.0;
            for (int r = 0; r < 3; ++r)
                Grows[v[q]][v[r]] += area * (gx[q] * gx[r] + gy[q] * gy[r]);
        }
    }
    for (int i = 0; i < ns; ++i)
        if (!(C[i] > 0)) return BTA_ERR_ARG;   // node in no triangle
    // --- K = G C^{-1} G and the union pattern ---------------------------------------------
    std::vector<std::map<int, double>> Krows(ns);
    for (int i = 0; i < ns; ++i)
        for (const auto& ik : Grows[i]) {
            const int k = ik.first;
            const double gik = ik.second / C[k];
            for (const auto& kj : Grows[k]) Krows[i][kj.first] += gik * kj.second;
        }
    std::vector<std::map<int, double>> U(ns);
    for (int i = 0; i < ns; ++i) {
        for (const auto& kv : Krows[i]) U[i][kv.first] = 0.0;
        for (const auto& kv : Grows[i]) U[i][kv.first] = 0.0;
        U[i][i] = 0.0;
    }
    Csr pat = to_csr(ns, U);
    const int nnz = (int)pat.col.size();
    std::vector<double> cval(nnz, 0.0), gval(nnz, 0.0), kval(nnz, 0.0);
    for (int i = 0; i < ns; ++i) {
        cval[find_pos(pat.rowptr, pat.col, i, i)] = C[i];
        for (const auto& kv : Grows[i]) gval[find_pos(pat.rowptr, pat.col, i, kv.first)] = kv.second;
        for (const auto& kv : Krows[i]) kval[find_pos(pat.rowptr, pat.col, i, kv.first)] = kv.second;
    }

    // --- observations: barycentric weights, Gram matrices, A^T y ---------------------------
    std::vector<double> gram((size_t)nt * nv * nnz, 0.0);
    std::vector<double> arrow((size_t)nt * nv * nr * ns, 0.0);
    std::vector<double> tip((size_t)nv * nr * nr, 0.0);
    std::vector<double> aty((size_t)N, 0.0);
    std::vector<double> stats(2 * nv, 0.0);
    std::vector<int> o_tv(m), o_s(3 * (size_t)m), o_gpos(9 * (size_t)m);
    std::vector<double> o_w(3 * (size_t)m), o_X((size_t)m * nr), o_y(m);
    for (int k = 0; k < m; ++k) {
        const int v = d->obs_var[k], t = d->obs_time[k], tr = d->obs_tri[k];
        if (v < 0 || v >= nv || t < 0 || t >= nt || tr < 0 || tr >= d->n_tri) return BTA_ERR_ARG;
        const double px = d->obs_xy[2 * k], py = d->obs_xy[2 * k + 1], yk = d->y[k];
        if (!std::isfinite(px) || !std::isfinite(py) || !std::isfinite(yk)) return BTA_ERR_NONFINITE;
        int s[3];
        double x[3], y[3];
        for (int q = 0; q < 3; ++q) {
            s[q] = d->tri[3 * tr + q];
            x[q] = d->nodes[2 * s[q]];
            y[q] = d->nodes[2 * s[q] + 1];
        }
        // barycentric coordinates: ratios of sub-triangle signed areas
        double det = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
        double w[3];
        for (int q = 0; q < 3; ++q) {
            int q1 = (q + 1) % 3, q2 = (q + 2) % 3;
            w[q] = ((x[q1] - px) * (y[q2] - py) - (x[q2] - px) * (y[q1] - py)) / det;
        }
        const size_t gbase = ((size_t)t * nv + v) * nnz;
        for (int q = 0; q < 3; ++q)
            for (int r = 0; r < 3; ++r) {
                int pos = find_pos(pat.rowptr, pat.col, s[q], s[r]);
                if (pos < 0) return BTA_ERR_ARG;   // cannot happen: triangle edges are in G
                gram[gbase + pos] += w[q] * w[r];
                o_gpos[9 * (size_t)k + 3 * q + r] = (int)(gbase + pos);
            }
        o_tv[k] = t * nv + v;
        o_y[k] = yk;
        for (int q = 0; q < 3; ++q) {
            o_s[3 * (size_t)k + q] = s[q];
            o_w[3 * (size_t)k + q] = w[q];
        }
        for (int r = 0; r < nr; ++r) o_X[(size_t)k * nr + r] = d->X[(size_t)k * nr + r];
        for (int r = 0; r < nr; ++r) {
            const double xr = d->X[(size_t)k * nr + r];
            for (int q = 0; q < 3; ++q)
                arrow[(((size_t)t * nv + v) * nr + r) * ns + s[q]] += xr * w[q];
            for (int r2 = 0; r2 < nr; ++r2)
                tip[((size_t)v * nr + r) * nr + r2] += xr * d->X[(size_t)k * nr + r2];
            aty[(size_t)n * b + (size_t)v * nr + r] += xr * yk;
        }
        for (int q = 0; q < 3; ++q) aty[(size_t)t * b + (size_t)v * ns + s[q]] += w[q] * yk;
        stats[v] += yk * yk;
        stats[nv + v] += 1.0;
    }

    std::vector<double> th0(dim_theta, 0.0);
    if (d->theta0) std::copy(d->theta0, d->theta0 + dim_theta, th0.begin());

    bta_model_s* M = new bta_model_s();
    std::memset(M, 0, sizeof(*M));
    M->nv = nv; M->ns = ns; M->nt = nt; M->nr = nr; M->m = m; M->dim_theta = dim_theta;
    M->n = n; M->b = b; M->a = a; M->N = N; M->nnz = nnz;
    M->beta_prec = d->beta_prior_prec;
    int rc = BTA_OK;
    if (rc == BTA_OK) rc = upload(&M->rowptr, pat.rowptr);
    if (rc == BTA_OK) rc = upload(&M->col, pat.col);
    if (rc == BTA_OK) rc = upload(&M->cval, cval);
    if (rc == BTA_OK) rc = upload(&M->gval, gval);
    if (rc == BTA_OK) rc = upload(&M->kval, kval);
    if (rc == BTA_OK) rc = upload(&M->gram, gram);
    if (rc == BTA_OK) rc = upload(&M->arrow, arrow);
    if (rc == BTA_OK) rc = upload(&M->tipgram, tip);
    if (rc == BTA_OK) rc = upload(&M->aty, aty);
    if (rc == BTA_OK) rc = upload(&M->theta0, th0);
    if (rc == BTA_OK) rc = upload(&M->var_stats, stats);
    if (rc == BTA_OK) rc = upload(&M->obs_tv, o_tv);
    if (rc == BTA_OK) rc = upload(&M->obs_s, o_s);
    if (rc == BTA_OK) rc = upload(&M->obs_w, o_w);
    if (rc == BTA_OK) rc = upload(&M->obs_gpos, o_gpos);
    if (rc == BTA_OK) rc = upload(&M->obs_X, o_X);
    if (rc == BTA_OK) rc = upload(&M->obs_y, o_y);
    if (rc != BTA_OK) {
        bta_model_destroy(M);
        return rc;
    }
    *out = M;
    return BTA_OK;
}

extern "C" int bta_model_destroy(bta_model_t M) {
    if (!M) return BTA_OK;
    void* ptrs[] = {M->rowptr, M->col, M->cval, M->gval, M->kval, M->gram, M->arrow,
                    M->tipgram, M->aty, M->theta0, M->var_stats, M->obs_tv, M->obs_s,
                    M->obs_w, M->obs_gpos, M->obs_X, M->obs_y};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete M;
    return BTA_OK;
}

extern "C" int bta_model_dims(bta_model_t M, int* n, int* b, int* a, int* dim_theta) {
    if (!M) return BTA_ERR_ARG;
    if (n) *n = M->n;
    if (b) *b = M->b;
    if (a) *a = M->a;
    if (dim_theta) *dim_theta = M->dim_theta;
    return BTA_OK;
}
