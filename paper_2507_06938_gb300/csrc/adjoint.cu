// Adjoint gradient of f_obj (Eq. 8) with respect to theta from the selected
// inverses, instead of the 2 dim(theta) extra evaluations of the central
// differences of Eq. 10.  For a Gaussian likelihood, with b = A^T D y,
// mu = Q_c^{-1} b and Sigma = Q^{-1} on the BTA pattern:
//   df/dtheta_k = dlog p(theta) + 1/2 tr(Sigma_p dQ_p) - 1/2 tr(Sigma_c dQ_c)
//                 - 1/2 y^T dD y + db^T mu - 1/2 mu^T dQ_c mu + 1/2 tr(D^{-1} dD)
// (d log|Q| = tr(Q^{-1} dQ); d mu = Q_c^{-1}(db - dQ_c mu)).  Every Q entry is
// a theta-dependent coefficient times a theta-free sparse matrix (C, G,
// G C^{-1} G, observation Gram matrices, identity of the fixed effects), so
// each trace splits into coefficient derivatives times theta-free inner
// products ("traces") <Sigma_block, M> over the sparsity pattern:
//   gather kernel   one CTA per (block, variable pair): <Sigma, C>, <Sigma, G>,
//                   <Sigma, G C^-1 G> and the Gram term, or the same with
//                   mu mu^T for the quadratic form (HBM gather)
//   arrow/tip kernel the fixed-effect blocks and the per-variable b^T mu parts
//   combine kernel  one thread per theta component: analytic derivatives of
//                   the coefficients (kappa, tau, rho, sigma, tau_eps, lambda)
// Diagonal blocks count once, the sub-diagonal and arrow blocks twice (the
// upper triangle mirrors them).

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "model_coef.cuh"

namespace {

// Per-matrix trace record (doubles): sp[blk][v][v'][3] for blk = 0..n-1
// (D_t) and n..2n-2 (B_t), then gram[t][v], arrow[t][v], tip[v][v'],
// tipgram[v], atydot[v].
struct TLayout {
    int n, nv;
    __host__ __device__ long long sp(int blk, int v, int w) const { return (((long long)blk * nv + v) * nv + w) * 3; }
    __host__ __device__ long long gram(int t, int v) const { return (long long)(2 * n - 1) * nv * nv * 3 + t * nv + v; }
    __host__ __device__ long long arrow(int t, int v) const { return gram(0, 0) + (long long)n * nv + t * nv + v; }
    __host__ __device__ long long tip(int v, int w) const { return arrow(0, 0) + (long long)n * nv + v * nv + w; }
    __host__ __device__ long long tipgram(int v) const { return tip(0, 0) + nv * nv + v; }
    __host__ __device__ long long atydot(int v) const { return tipgram(0) + nv + v; }
    __host__ __device__ long long size() const { return atydot(0) + nv; }
};

struct GatherArgs {
    int n, b, a, ns, nv, nr, nnz;
    long long N;
    const int* rowptr;
    const int* col;
    const double* cval;
    const double* gval;
    const double* kval;
    const double* gram;
    const double* arrow;
    const double* tipgram;
    const double* aty;
    // Sigma mode: selected-inverse blocks of matrix z at S* + z s*
    const double* SD;
    const double* SB;
    const double* SR;
    const double* ST;
    long long sD, sB, sR, sT;
    // mu mode (SD == nullptr): vectors mu_z at mu + z N
    const double* mu;
    double* out;      // record of matrix z at out + z rec
    long long rec;
    TLayout lay;
};

__device__ __forceinline__ double block_sum_d(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (w == 0) {
        s = (lane < (int)(blockDim.x / 32)) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;
}

// grid: x = block (0..2n-2), y = v * nv + v', z = matrix
__global__ void __launch_bounds__(256) trace_spatial_kernel(GatherArgs p) {
    __shared__ double red[32];
    const int blk = blockIdx.x, v = blockIdx.y / p.nv, w = blockIdx.y % p.nv, z = blockIdx.z;
    const bool diag = blk < p.n;
    const int t = diag ? blk : blk - p.n;   // column time block
    const int tr = diag ? t : t + 1;        // row time block
    const long long bb = (long long)p.b * p.b;
    const double* blockS = nullptr;
    const double* mu = nullptr;
    if (p.SD) blockS = diag ? p.SD + z * p.sD + t * bb : p.SB + z * p.sB + t * bb;
    else mu = p.mu + z * p.N;
    const bool with_gram = diag && v == w;
    const double* gram = p.gram + ((long long)t * p.nv + v) * p.nnz;
    double ac = 0, ag = 0, ak = 0, aG = 0;
    for (int sc = threadIdx.x; sc < p.ns; sc += blockDim.x) {
        // column (w, sc) of the block; rows (v, s) for s in the pattern of column sc
        const long long colj = (long long)w * p.ns + sc;
        const double mucol = mu ? mu[(long long)t * p.b + colj] : 0.0;
        for (int q = p.rowptr[sc]; q < p.rowptr[sc + 1]; ++q) {
            const int s = p.col[q];
            const long long rowi = (long long)v * p.ns + s;
            const double e = blockS ? blockS[rowi + colj * p.b] : mu[(long long)tr * p.b + rowi] * mucol;
            ac = fma(e, p.cval[q], ac);
            ag = fma(e, p.gval[q], ag);
            ak = fma(e, p.kval[q], ak);
            if (with_gram) aG = fma(e, gram[q], aG);
        }
    }
    double* out = p.out + z * p.rec;
    const double sc_ = block_sum_d(ac, red);
    const double sg = block_sum_d(ag, red);
    const double sk = block_sum_d(ak, red);
    const double sG = block_sum_d(aG, red);
    if (threadIdx.x == 0) {
        const long long o = p.lay.sp(blk, v, w);
        out[o] = sc_;
        out[o + 1] = sg;
        out[o + 2] = sk;
        if (with_gram) out[p.lay.gram(t, v)] = sG;
    }
}

// grid: x = n*nv arrow records, then 1 tip record, then nv b^T mu parts; y = matrix
__global__ void __launch_bounds__(256) trace_fixed_kernel(GatherArgs p) {
    __shared__ double red[32];
    const int z = blockIdx.y;
    const int nv = p.nv, nr = p.nr, a = p.a;
    const long long nb = (long long)p.n * p.b;
    const double* mu = p.SD ? nullptr : p.mu + z * p.N;
    double* out = p.out + z * p.rec;
    const int x = blockIdx.x;
    if (x < p.n * nv) {
        // <Sigma_{tip,t}^{vv}, Arrow_{t,v}> = sum_{r,s} E[(v,r),(t,v,s)] arrow[t][v][r][s]
        const int t = x / nv, v = x % nv;
        double acc = 0.0;
        for (int e = threadIdx.x; e < nr * p.ns; e += blockDim.x) {
            const int r = e / p.ns, s = e % p.ns;
            const int row = v * nr + r;
            const long long colj = (long long)v * p.ns + s;
            const double E = mu ? mu[nb + row] * mu[(long long)t * p.b + colj]
                                : p.SR[z * p.sR + (long long)t * a * p.b + colj * a + row];
            acc = fma(E, p.arrow[(((long long)t * nv + v) * nr + r) * p.ns + s], acc);
        }
        const double sum = block_sum_d(acc, red);
        if (threadIdx.x == 0) out[p.lay.arrow(t, v)] = sum;
    } else if (x == p.n * nv) {
        // tip[v][w] = sum_r E[(v,r),(w,r)];  tipgram[v] = sum_{r,r'} E[(v,r),(v,r')] tipgram[v][r][r']
        for (int e = threadIdx.x; e < nv * nv + nv; e += blockDim.x) {
            if (e < nv * nv) {
                const int v = e / nv, w = e % nv;
                double acc = 0.0;
                for (int r = 0; r < nr; ++r) {
                    const int i = v * nr + r, j = w * nr + r;
                    acc += mu ? mu[nb + i] * mu[nb + j] : p.ST[z * p.sT + (long long)j * a + i];
                }
                out[p.lay.tip(v, w)] = acc;
            } else {
                const int v = e - nv * nv;
                double acc = 0.0;
                for (int r = 0; r < nr; ++r)
                    for (int r2 = 0; r2 < nr; ++r2) {
                        const int i = v * nr + r, j = v * nr + r2;
                        const double E = mu ? mu[nb + i] * mu[nb + j] : p.ST[z * p.sT + (long long)j * a + i];
                        acc += E * p.tipgram[((long long)v * nr + r) * nr + r2];
                    }
                out[p.lay.tipgram(v)] = acc;
            }
        }
    } else {
        // b^T mu restricted to variable v (unscaled A^T y of that variable)
        const int v = x - p.n * nv - 1;
        double acc = 0.0;
        if (mu) {
            for (long long e = threadIdx.x; e < (long long)p.n * p.ns + nr; e += blockDim.x) {
                long long i;
                if (e < (long long)p.n * p.ns) {
                    const long long t = e / p.ns, s = e % p.ns;
                    i = t * p.b + (long long)v * p.ns + s;
                } else {
                    i = nb + (long long)v * nr + (e - (long long)p.n * p.ns);
                }
                acc = fma(p.aty[i], mu[i], acc);
            }
        }
        const double sum = block_sum_d(acc, red);
        if (threadIdx.x == 0) out[p.lay.atydot(v)] = sum;
    }
}

struct CombineArgs {
    int n, nv, nr, nt, dim;
    double beta_prec;
    const double* params;     // slot j at params + j BTA_PSTRIDE
    const double* theta;      // slot j at theta + j dim
    const double* theta0;
    const double* var_stats;  // ||y_v||^2, m_v
    const double* Tp;         // trace record of Q_p of slot j at Tp + j rec
    const double* Tc;         // ... of Q_c
    const double* Tm;         // mu mu^T record of slot j
    long long rec;
    TLayout lay;
    double* grad;             // slot j at grad + j dim
};

// blockIdx.x = slot j, threadIdx.x = theta component k
__global__ void adjoint_combine_kernel(CombineArgs p) {
    const int j = blockIdx.x, k = threadIdx.x;
    if (k >= p.dim) return;
    const int nv = p.nv;
    const double* P = p.params + (long long)j * BTA_PSTRIDE;
    const double* lam = P + 5 * nv;
    const double* Tp = p.Tp + j * p.rec;
    const double* Tc = p.Tc + j * p.rec;
    const double* Tm = p.Tm + j * p.rec;
    const int uk = k < 4 * nv ? k / 4 : -1;      // variable of the component
    const int which = k < 4 * nv ? k % 4 : 4;    // 0 range_s, 1 range_t, 2 sigma, 3 tau_eps, 4 lambda
    int lr = -1, lc = -1;
    if (which == 4) lambda_position(nv, k - 4 * nv, &lr, &lc);
    // derivative of c_u(v,w) = Minv[u][v] Minv[u][w] / sigma_u^2
    auto dc = [&](int u, int v, int w) -> double {
        const double s2 = P[5 * u + 3] * P[5 * u + 3];
        const double mv = minv_entry(lam, nv, u, v), mw = minv_entry(lam, nv, u, w);
        if (which == 2) return u == uk ? -2.0 * mv * mw / s2 : 0.0;
        if (which == 4) {
            const double dmv = (u == lr && v == lc) ? -1.0 : 0.0;
            const double dmw = (u == lr && w == lc) ? -1.0 : 0.0;
            return (dmv * mw + mv * dmw) / s2;
        }
        return 0.0;
    };
    double g = -(p.theta[(long long)j * p.dim + k] - p.theta0[k]);
    // spatio-temporal blocks
    for (int blk = 0; blk < 2 * p.n - 1; ++blk) {
        const bool diag = blk < p.n;
        const int t = diag ? blk : blk - p.n, tr = diag ? t : t + 1;
        const double wgt = diag ? 1.0 : 2.0;
        for (int v = 0; v < nv; ++v)
            for (int w = 0; w < nv; ++w) {
                double dcoef[3] = {0.0, 0.0, 0.0};
                for (int u = 0; u < nv; ++u) {
                    const double kap = P[5 * u], tau = P[5 * u + 1], rho = P[5 * u + 2], sig = P[5 * u + 3];
                    const double c = minv_entry(lam, nv, u, v) * minv_entry(lam, nv, u, w) / (sig * sig);
                    const double t2 = tau * tau, k2 = kap * kap;
                    const double spat[3] = {t2 * k2 * k2, 2.0 * t2 * k2, t2};
                    const double qt = ar1_entry(rho, p.nt, tr, t);
                    if (which == 0 && u == uk) {
                        dcoef[0] += c * qt * (-2.0 * spat[0]);
                        dcoef[2] += c * qt * (2.0 * spat[2]);
                    } else if (which == 1 && u == uk) {
                        const double dq = ar1_drho(rho, p.nt, tr, t) * (-rho * log(rho));
                        for (int q = 0; q < 3; ++q) dcoef[q] += c * dq * spat[q];
                    } else if (which == 2 || which == 4) {
                        const double d = dc(u, v, w);
                        for (int q = 0; q < 3; ++q) dcoef[q] += d * qt * spat[q];
                    }
                }
                const long long o = p.lay.sp(blk, v, w);
                for (int q = 0; q < 3; ++q)
                    g += wgt * dcoef[q] * (0.5 * Tp[o + q] - 0.5 * Tc[o + q] - 0.5 * Tm[o + q]);
            }
    }
    // fixed-effect prior (tip): sum_u c_u(v,w) p_beta on the diagonal of each (v,w) block
    if (which == 2 || which == 4)
        for (int v = 0; v < nv; ++v)
            for (int w = 0; w < nv; ++w) {
                double d = 0.0;
                for (int u = 0; u < nv; ++u) d += dc(u, v, w);
                const long long o = p.lay.tip(v, w);
                g += d * p.beta_prec * (0.5 * Tp[o] - 0.5 * Tc[o] - 0.5 * Tm[o]);
            }
    // observation terms: dQ_c = tau_eps_u (Gram, arrow, tip Gram of variable u), dD, db
    if (which == 3) {
        const double te = P[5 * uk + 4];
        double tc = 0.0, tm = 0.0;
        for (int t = 0; t < p.n; ++t) {
            tc += Tc[p.lay.gram(t, uk)] + 2.0 * Tc[p.lay.arrow(t, uk)];
            tm += Tm[p.lay.gram(t, uk)] + 2.0 * Tm[p.lay.arrow(t, uk)];
        }
        tc += Tc[p.lay.tipgram(uk)];
        tm += Tm[p.lay.tipgram(uk)];
        g += -0.5 * te * tc - 0.5 * te * tm;
        g += -0.5 * te * p.var_stats[uk] + te * Tm[p.lay.atydot(uk)] + 0.5 * p.var_stats[nv + uk];
    }
    p.grad[(long long)j * p.dim + k] = g;
}

}  // namespace

long long adjoint_record_size(int n, int nv) { return TLayout{n, nv}.size(); }

// Traces of the matrices m0 .. m0+cnt-1 (selected inverses, or mu mu^T of the
// Q_c vectors when mu_mode) into out (records of `rec` doubles).
static int gather_traces(bta_ctx_t ctx, bta_model_t m, int m0, int cnt, bool mu_mode, double* out, long long rec,
                         cudaStream_t s) {
    GatherArgs p;
    p.n = ctx->n; p.b = ctx->b; p.a = ctx->a; p.ns = m->ns; p.nv = m->nv; p.nr = m->nr; p.nnz = m->nnz;
    p.N = ctx->N;
    p.rowptr = m->rowptr; p.col = m->col; p.cval = m->cval; p.gval = m->gval; p.kval = m->kval;
    p.gram = m->gram; p.arrow = m->arrow; p.tipgram = m->tipgram; p.aty = m->aty;
    const BtaStore& S = ctx->S;
    if (!mu_mode) {
        p.SD = S.D + m0 * S.sD; p.SB = S.B + m0 * S.sB; p.SR = S.R + m0 * S.sR; p.ST = S.T + m0 * S.sT;
        p.sD = S.sD; p.sB = S.sB; p.sR = S.sR; p.sT = S.sT;
        p.mu = nullptr;
    } else {
        p.SD = p.SB = p.SR = p.ST = nullptr;
        p.sD = p.sB = p.sR = p.sT = 0;
        p.mu = vec_row(ctx, VEC_MU, m0);
    }
    p.out = out;
    p.rec = rec;
    p.lay = TLayout{ctx->n, m->nv};
    trace_spatial_kernel<<<dim3(2 * ctx->n - 1, m->nv * m->nv, cnt), 256, 0, s>>>(p);
    BTA_LAUNCH_CHECK();
    if (m->nr > 0 || mu_mode) {
        trace_fixed_kernel<<<dim3(ctx->n * m->nv + 1 + m->nv, cnt), 256, 0, s>>>(p);
        BTA_LAUNCH_CHECK();
    }
    return BTA_OK;
}

extern "C" int bta_fobj_grad(bta_ctx_t ctx, bta_model_t m, const double* thetas_dev, int n_theta, double* f_out_dev,
                             double* grad_out_dev) {
    if (!ctx || !m || !thetas_dev || !f_out_dev || !grad_out_dev || n_theta < 1) return BTA_ERR_ARG;
    if (m->n != ctx->n || m->b != ctx->b || m->a != ctx->a || m->nv > BTA_MAX_NV || m->dim_theta > 1024)
        return BTA_ERR_ARG;
    cudaStream_t s = ctx->stream;
    const int B = ctx->batch;
    const long long rec = adjoint_record_size(ctx->n, m->nv);
    if (!ctx->adj) {
        // records: 2B matrices (Sigma traces) + B slots (mu mu^T)
        cudaError_t e = cudaMalloc((void**)&ctx->adj, (size_t)3 * B * rec * sizeof(double));
        if (e != cudaSuccess) {
            ctx->adj = nullptr;
            return bta_cuda_fail(e);
        }
        BTA_CUDA_TRY(cudaMemsetAsync(ctx->adj, 0, (size_t)3 * B * rec * sizeof(double), s));
    }
    BTA_TRY(ensure_sigma(ctx));
    for (int r0 = 0; r0 < n_theta; r0 += B) {
        const int cnt = std::min(B, n_theta - r0);
        BTA_TRY(fobj_eval(ctx, m, thetas_dev + (long long)r0 * m->dim_theta, cnt, f_out_dev + r0, nullptr));
        if (cnt == B) {
            BTA_TRY(selinv_impl(ctx, 0, 2 * B, s));
        } else {
            BTA_TRY(selinv_impl(ctx, 0, cnt, s));
            BTA_TRY(selinv_impl(ctx, B, cnt, s));
        }
        BTA_TRY(prof_phase(ctx, 4, s));
        double* Tp = ctx->adj;
        double* Tc = ctx->adj + (long long)B * rec;
        double* Tm = ctx->adj + 2LL * B * rec;
        BTA_TRY(gather_traces(ctx, m, 0, cnt, false, Tp, rec, s));
        BTA_TRY(gather_traces(ctx, m, B, cnt, false, Tc, rec, s));
        BTA_TRY(gather_traces(ctx, m, B, cnt, true, Tm, rec, s));
        CombineArgs c;
        c.n = ctx->n; c.nv = m->nv; c.nr = m->nr; c.nt = m->nt; c.dim = m->dim_theta;
        c.beta_prec = m->beta_prec;
        c.params = ctx->params;
        c.theta = thetas_dev + (long long)r0 * m->dim_theta;
        c.theta0 = m->theta0;
        c.var_stats = m->var_stats;
        c.Tp = Tp; c.Tc = Tc; c.Tm = Tm; c.rec = rec;
        c.lay = TLayout{ctx->n, m->nv};
        c.grad = grad_out_dev + (long long)r0 * m->dim_theta;
        const int threads = ((m->dim_theta + 31) / 32) * 32;
        adjoint_combine_kernel<<<cnt, threads, 0, s>>>(c);
        BTA_LAUNCH_CHECK();
        BTA_TRY(prof_phase(ctx, 5, s));
    }
    return BTA_OK;
}
