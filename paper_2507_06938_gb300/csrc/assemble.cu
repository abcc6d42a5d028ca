// Device assembly of the BTA blocks of Q_p and Q_c (Sections II-A, IV-B, IV-F).
//
// Every block entry is a theta-dependent linear combination of theta-free
// sparse data held by the model:
//   D_t[(v,s),(v',s')] = sum_u c_u(v,v') Qt_u[t,t] (alpha_u C + beta_u G + gamma_u K)[s,s']
//                        + [Q_c, v = v'] tau_eps_v Gram_{t,v}[s,s']
//   B_t[(v,s),(v',s')] = sum_u c_u(v,v') Qt_u[t+1,t] (alpha_u C + beta_u G + gamma_u K)[s,s']
//   R_t[(v,r),(v',s')] = [Q_c, v = v'] tau_eps_v Arrow_{t,v}[r,s']
//   T[(v,r),(v',r')]   = sum_u c_u(v,v') p_beta [r = r'] + [Q_c, v = v'] tau_eps_v Tip_v[r,r']
// with K = G C^{-1} G, alpha_u = tau_u^2 kappa_u^4, beta_u = 2 tau_u^2 kappa_u^2,
// gamma_u = tau_u^2 (SPDE precision), c_u(v,v') = Minv[u,v] Minv[u,v'] / sigma_u^2
// (Eq. 11) and Qt_u the stationary AR(1) precision.  One CTA builds one column
// of one D/B block in shared memory (zero fill + sparse scatter) and writes it
// out with coalesced stores: the kernel is bound by the HBM write of the
// dense blocks.

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "model_coef.cuh"

namespace {

constexpr int ASM_THREADS = 256;

struct AsmArgs {
    int n, b, a, ns, nv, nr, nt, nnz;
    int m0, batch;           // matrices m0 + blockIdx.z; kind = m / batch, slot = m % batch
    long long sD, sB, sR, sT;
    const int* rowptr;
    const int* col;
    const double* cval;
    const double* gval;
    const double* kval;
    const double* gram;
    const double* arrow;
    const double* tipgram;
    long long gs, as, ts;    // per-slot strides of gram / arrow / tipgram (0: the model's, shared)
    const double* params;    // parameter slots, pstride apart (0: one vector for all)
    long long pstride;
    double beta_prec;
    double* D;
    double* B;
    double* R;
    double* T;
};

// grid: x = column j (0..b-1), y = block: 0..n-1 -> D_y, n..2n-2 -> B_{y-n},
// z = matrix
__global__ void __launch_bounds__(ASM_THREADS) assemble_db_kernel(AsmArgs p) {
    extern __shared__ double colbuf[];   // b doubles
    __shared__ double coef[BTA_MAX_NV][3];
    __shared__ double obsw[BTA_MAX_NV];
    const int mat = p.m0 + blockIdx.z;
    const int with_obs = mat / p.batch;           // 0: Q_p, 1: Q_c
    const double* params = p.params + (long long)(mat % p.batch) * p.pstride;
    const int j = blockIdx.x;
    const int blk = blockIdx.y;
    const bool diag = blk < p.n;
    const int t = diag ? blk : blk - p.n;              // column time index
    const int trow = diag ? t : t + 1;                 // row time index
    const int vp = j / p.ns, sp = j % p.ns;
    const int nv = p.nv;
    const double* lam = params + 5 * nv;
    if (threadIdx.x < nv) {
        const int v = threadIdx.x;
        double ca = 0, cb = 0, cg = 0;
        for (int u = 0; u < nv; ++u) {
            const double* pu = params + 5 * u;
            const double kappa = pu[0], tau = pu[1], rho = pu[2], sigma = pu[3];
            double c = minv_entry(lam, nv, u, v) * minv_entry(lam, nv, u, vp) / (sigma * sigma);
            if (c == 0.0) continue;
            c *= ar1_entry(rho, p.nt, trow, t);
            const double t2 = tau * tau, k2 = kappa * kappa;
            ca += c * t2 * k2 * k2;
            cb += c * 2.0 * t2 * k2;
            cg += c * t2;
        }
        coef[v][0] = ca;
        coef[v][1] = cb;
        coef[v][2] = cg;
        obsw[v] = (with_obs && diag && v == vp) ? params[5 * v + 4] : 0.0;
    }
    for (int r = threadIdx.x; r < p.b; r += ASM_THREADS) colbuf[r] = 0.0;
    __syncthreads();
    const int r0 = p.rowptr[sp], r1 = p.rowptr[sp + 1];
    const int len = r1 - r0;
    const double* gram = p.gram + (mat % p.batch) * p.gs + ((size_t)t * nv + vp) * p.nnz;
    for (int e = threadIdx.x; e < len * nv; e += ASM_THREADS) {
        const int v = e / len;
        const int q = r0 + (e - v * len);
        const int s = p.col[q];
        double val = coef[v][0] * p.cval[q] + coef[v][1] * p.gval[q] + coef[v][2] * p.kval[q];
        if (obsw[v] != 0.0) val += obsw[v] * gram[q];
        colbuf[v * p.ns + s] = val;
    }
    __syncthreads();
    double* out = diag ? p.D + mat * p.sD + (size_t)t * p.b * p.b : p.B + mat * p.sB + (size_t)t * p.b * p.b;
    out += (size_t)j * p.b;
    for (int r = threadIdx.x; r < p.b; r += ASM_THREADS) out[r] = colbuf[r];
}

// R_t and T: one thread per entry.  Entries 0..n*a*b-1 are R (column-major
// per block), then a*a entries of T; blockIdx.y = matrix.
__global__ void assemble_rt_kernel(AsmArgs p) {
    const long long total = (long long)p.n * p.a * p.b + (long long)p.a * p.a;
    const int nv = p.nv, nr = p.nr;
    const int mat = p.m0 + blockIdx.y;
    const int with_obs = mat / p.batch;
    const double* params = p.params + (long long)(mat % p.batch) * p.pstride;
    const double* lam = params + 5 * nv;
    double* R = p.R + mat * p.sR;
    double* T = p.T + mat * p.sT;
    const double* arrow = p.arrow + (mat % p.batch) * p.as;
    const double* tipgram = p.tipgram + (mat % p.batch) * p.ts;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long nab = (long long)p.n * p.a * p.b;
        if (idx < nab) {
            const int t = (int)(idx / ((long long)p.a * p.b));
            const int rem = (int)(idx - (long long)t * p.a * p.b);
            const int colj = rem / p.a, row = rem % p.a;
            const int v = row / nr, r = row % nr;
            const int vp = colj / p.ns, s = colj % p.ns;
            double val = 0.0;
            if (with_obs && v == vp)
                val = params[5 * v + 4] * arrow[(((size_t)t * nv + v) * nr + r) * p.ns + s];
            R[idx] = val;
        } else {
            const int e = (int)(idx - nab);
            const int colj = e / p.a, row = e % p.a;
            const int v = row / nr, r = row % nr;
            const int vp = colj / nr, rp = colj % nr;
            double val = 0.0;
            if (r == rp) {
                for (int u = 0; u < nv; ++u) {
                    const double sigma = params[5 * u + 3];
                    val += minv_entry(lam, nv, u, v) * minv_entry(lam, nv, u, vp) / (sigma * sigma);
                }
                val *= p.beta_prec;
            }
            if (with_obs && v == vp)
                val += params[5 * v + 4] * tipgram[((size_t)v * nr + r) * nr + rp];
            T[e] = val;
        }
    }
}

// blockIdx.x = slot: theta + slot dim_theta -> params + slot BTA_PSTRIDE
__global__ void theta_to_params_kernel(const double* theta, int nv, int dim_theta, double* params) {
    theta += (long long)blockIdx.x * dim_theta;
    params += (long long)blockIdx.x * BTA_PSTRIDE;
    const int i = threadIdx.x;
    if (i < nv) {
        const double range_s = exp(theta[4 * i + 0]);
        const double range_t = exp(theta[4 * i + 1]);
        const double kappa = sqrt(8.0) / range_s;
        params[5 * i + 0] = kappa;
        params[5 * i + 1] = sqrt(1.0 / (4.0 * M_PI * kappa * kappa));
        params[5 * i + 2] = exp(-1.0 / range_t);
        params[5 * i + 3] = exp(theta[4 * i + 2]);
        params[5 * i + 4] = exp(theta[4 * i + 3]);
    }
    const int nl = nv * (nv - 1) / 2;
    if (i < nl) params[5 * nv + i] = theta[4 * nv + i];
}

}  // namespace

int theta_to_params_impl(bta_model_t m, const double* theta, int count, double* params, cudaStream_t s) {
    if (count <= 0) return BTA_OK;
    theta_to_params_kernel<<<count, 64, 0, s>>>(theta, m->nv, m->dim_theta, params);
    BTA_LAUNCH_CHECK();
    return BTA_OK;
}

static int assemble_run(bta_ctx_t ctx, bta_model_t m, const double* params, long long pstride, int m0, int count,
                        cudaStream_t s, const ObsWeights* w = nullptr) {
    if (count <= 0) return BTA_OK;
    AsmArgs p;
    p.n = ctx->n; p.b = ctx->b; p.a = ctx->a;
    p.ns = m->ns; p.nv = m->nv; p.nr = m->nr; p.nt = m->nt; p.nnz = m->nnz;
    p.m0 = m0; p.batch = ctx->batch;
    p.rowptr = m->rowptr; p.col = m->col;
    p.cval = m->cval; p.gval = m->gval; p.kval = m->kval; p.gram = m->gram;
    p.arrow = m->arrow; p.tipgram = m->tipgram;
    p.gs = p.as = p.ts = 0;
    if (w) {
        // observation terms weighted per observation and slot (non-Gaussian likelihoods)
        p.gram = w->gram; p.arrow = w->arrow; p.tipgram = w->tip;
        p.gs = w->gram_stride; p.as = w->arrow_stride; p.ts = w->tip_stride;
    }
    p.params = params;
    p.pstride = pstride;
    p.beta_prec = m->beta_prec;
    const BtaStore& Q = ctx->Q;
    p.D = Q.D; p.B = Q.B; p.R = Q.R; p.T = Q.T;
    p.sD = Q.sD; p.sB = Q.sB; p.sR = Q.sR; p.sT = Q.sT;
    const size_t smem = (size_t)p.b * sizeof(double);
    BTA_TRY(ensure_dyn_smem((const void*)assemble_db_kernel, (int)smem));
    dim3 grid(p.b, 2 * p.n - 1, count);
    assemble_db_kernel<<<grid, ASM_THREADS, smem, s>>>(p);
    BTA_LAUNCH_CHECK();
    const long long total = (long long)p.n * p.a * p.b + (long long)p.a * p.a;
    if (total > 0) {
        int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 16);
        assemble_rt_kernel<<<dim3(blocks, count), 256, 0, s>>>(p);
        BTA_LAUNCH_CHECK();
    }
    for (int k = m0; k < m0 + count; ++k) ctx->factored[k] = 0;
    return BTA_OK;
}

int assemble_impl(bta_ctx_t ctx, bta_model_t m, const double* params, int m0, int count, cudaStream_t s) {
    return assemble_run(ctx, m, params, BTA_PSTRIDE, m0, count, s);
}

int assemble_weighted_impl(bta_ctx_t ctx, bta_model_t m, const double* params, int m0, int count, cudaStream_t s,
                           const ObsWeights& w) {
    return assemble_run(ctx, m, params, BTA_PSTRIDE, m0, count, s, &w);
}

extern "C" int bta_assemble(bta_ctx_t ctx, bta_model_t m, const double* params_dev, int which) {
    if (!ctx || !m || !params_dev) return BTA_ERR_ARG;
    if (m->n != ctx->n || m->b != ctx->b || m->a != ctx->a || m->nv > BTA_MAX_NV) return BTA_ERR_ARG;
    const int mat = storage_index(ctx, which);
    if (mat < 0) return BTA_ERR_ARG;
    return assemble_run(ctx, m, params_dev, 0, mat, 1, ctx->stream);
}

extern "C" int bta_theta_to_params(bta_ctx_t ctx, bta_model_t m, const double* theta_dev, double* params_dev) {
    if (!ctx || !m || !theta_dev || !params_dev) return BTA_ERR_ARG;
    return theta_to_params_impl(m, theta_dev, 1, params_dev, ctx->stream);
}
