// nf_adjoint.cu -- discrete adjoint of the RK4 map of nf_rk4_advance (matrix-free).
//
// One RK4 step (b = (1, 2, 2, 1) / 6, c = (1/2, 1/2, 1) for U_{s+1} = u + c_s dt k_s)
// is reversed stage by stage:
//     nu_4 = dt b_4 lam,                mu_s = J(U_s)^T nu_s = -nu_s + q o f'(U_s) o (W nu_s),
//     nu_s = dt b_s lam + c_s dt mu_{s+1}  (s = 3, 2, 1),
//     lam <- lam + mu_1 + mu_2 + mu_3 + mu_4,
// with W symmetric because the kernel is radial.  Kernel-parameter gradients add
//     <nu_s, (d_theta W) (q o f(U_s))>,  d w / dA1 = e1, d w / ds1 = 2 A1 r^2 e1 / s1^3,
//     d w / dA2 = -e2,  d w / ds2 = -2 A2 r^2 e2 / s2^3.
// The adjoint pair kernel computes, per row i and in one pass over the columns,
//     sum_j e1 nu_j, sum_j e2 nu_j, sum_j e1 g_j, sum_j r^2 e1 g_j, sum_j e2 g_j,
//     sum_j r^2 e2 g_j   (two SFU exponentials per pair, six FP32 accumulators),
// staged like the forward kernel (TMA bulk tiles of x and of (nu, g) pairs).  The
// epilogue applies the recurrences, writes per-row gradient contributions and prepares
// (nu, g) of the next stage; a fixed-order reduction accumulates the parameter
// gradients in FP64.  Stage inputs are recomputed segment by segment from checkpoints.
#include "nf_internal.cuh"

#include <algorithm>

namespace nfi {

constexpr int AD_THREADS = 256;
constexpr int AD_WARPS = AD_THREADS / 32;
constexpr int AD_TJ = 512;
constexpr int AD_R = 2;  // rows per warp (6 accumulators each)
static_assert(kNodePad % AD_TJ == 0, "tile must divide the node padding");

struct AdSmem {
    float4 xs[2][AD_TJ];
    float2 vg[2][AD_TJ];
    uint64_t bar[2];
};

// partial layout: [6][splits][B][n_pad]
__global__ void __launch_bounds__(AD_THREADS)
adj_pair_kernel(const float4 *__restrict__ x4, const float2 *__restrict__ vg, int64_t n_pad, int B, int b,
                int64_t jchunk, float c1, float c2, float *__restrict__ partial, int *__restrict__ err) {
    __shared__ __align__(128) AdSmem sm;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int split = blockIdx.y, nsplit = gridDim.y;
    const int64_t j0 = (int64_t)split * jchunk, j1 = min(n_pad, j0 + jchunk);
    const int ntiles = (int)((j1 - j0) / AD_TJ);
    const int64_t row0 = ((int64_t)blockIdx.x * AD_WARPS + warp) * AD_R;
    const float2 *vgb = vg + (int64_t)b * n_pad;
    constexpr uint32_t kTileBytes = AD_TJ * 16 + AD_TJ * 8;
    if (tid == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](int t) {
        const int buf = t & 1;
        const int64_t jt = j0 + (int64_t)t * AD_TJ;
        mbar_arrive_expect_tx(&sm.bar[buf], kTileBytes);
        bulk_g2s(sm.xs[buf], x4 + jt, AD_TJ * 16, &sm.bar[buf]);
        bulk_g2s(sm.vg[buf], vgb + jt, AD_TJ * 8, &sm.bar[buf]);
    };
    if (tid == 0) {
        if (ntiles > 0) issue(0);
        if (ntiles > 1) issue(1);
    }
    float xi[AD_R], yi[AD_R], zi[AD_R];
    float acc[AD_R][6];
#pragma unroll
    for (int r = 0; r < AD_R; ++r) {
        const float4 p = x4[row0 + r];
        xi[r] = p.x;
        yi[r] = p.y;
        zi[r] = p.z;
#pragma unroll
        for (int a = 0; a < 6; ++a) acc[r][a] = 0.f;
    }
    bool timed_out = false;
    for (int t = 0; t < ntiles; ++t) {
        const int buf = t & 1;
        const bool ok = mbar_wait_bounded(&sm.bar[buf], (uint32_t)((t >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        if (tid == 0 && t >= 1 && t + 1 < ntiles) issue(t + 1);
#pragma unroll 2
        for (int jj = lane; jj < AD_TJ; jj += 32) {
            const float4 xj = sm.xs[buf][jj];
            const float2 p = sm.vg[buf][jj];  // (nu_j, g_j)
#pragma unroll
            for (int r = 0; r < AD_R; ++r) {
                const float dx = xi[r] - xj.x, dy = yi[r] - xj.y, dz = zi[r] - xj.z;
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                const float e1 = ex2_sfu(r2 * c1), e2 = ex2_sfu(r2 * c2);
                const float e1g = e1 * p.y, e2g = e2 * p.y;
                acc[r][0] = fmaf(e1, p.x, acc[r][0]);
                acc[r][1] = fmaf(e2, p.x, acc[r][1]);
                acc[r][2] += e1g;
                acc[r][3] = fmaf(r2, e1g, acc[r][3]);
                acc[r][4] += e2g;
                acc[r][5] = fmaf(r2, e2g, acc[r][5]);
            }
        }
    }
    if (timed_out) {
        if (tid == 0) {
            set_dev_error(err, DEV_TIMEOUT);
            for (int bb = 0; bb < 2; ++bb) (void)mbar_wait_bounded(&sm.bar[bb], 0), (void)mbar_wait_bounded(&sm.bar[bb], 1);
        }
        return;
    }
    const int64_t plane = (int64_t)nsplit * B * n_pad;
#pragma unroll
    for (int r = 0; r < AD_R; ++r)
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            const float v = warp_sum(acc[r][a]);
            if (lane == 0) partial[a * plane + ((int64_t)split * B + b) * n_pad + row0 + r] = v;
        }
}

__device__ __forceinline__ float sigmoid_rate(float u, float beta, float theta) {
    return 1.0f / (1.0f + expf(-beta * (u - theta)));
}

// vg[b, i] = (dt b4 lam_i, q_i f(U_i))  -- entering the last stage of a step
__global__ void adj_prep_kernel(const float *__restrict__ lam, const float *__restrict__ U, const float *__restrict__ q,
                                const float *__restrict__ beta, const float *__restrict__ theta, int64_t n,
                                int64_t n_pad, int B, float dtb4, float2 *__restrict__ vg) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)B * n) return;
    const int b = (int)(idx / n);
    const int64_t i = idx - (int64_t)b * n;
    vg[(int64_t)b * n_pad + i] = make_float2(dtb4 * lam[idx], q[i] * sigmoid_rate(U[idx], beta[b], theta[b]));
}

struct AdjEpiArgs {
    const float *partial;
    int splits;
    int64_t n, n_pad;
    int B;
    int stg;                 // 0..3 (stage s = stg + 1)
    const float *Ucur;       // U_s
    const float *Uprev;      // U_{s-1} (stg > 0), U_4 of the previous step (stg == 0), or null
    float *lam, *acc;
    float2 *vg;
    float *contrib;          // [B][4][n]
    const float *q, *beta, *theta;
    float A1, A2, dA1c, dA2c;  // dA1c = 2 A1 / s1^3, dA2c = 2 A2 / s2^3
    float dt;
};

__global__ void adj_epilogue_kernel(AdjEpiArgs a) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)a.B * a.n) return;
    const int b = (int)(idx / a.n);
    const int64_t i = idx - (int64_t)b * a.n;
    const int64_t plane = (int64_t)a.splits * a.B * a.n_pad;
    float s6[6] = {0, 0, 0, 0, 0, 0};
    for (int sp = 0; sp < a.splits; ++sp) {
        const int64_t off = ((int64_t)sp * a.B + b) * a.n_pad + i;
#pragma unroll
        for (int k = 0; k < 6; ++k) s6[k] += a.partial[k * plane + off];
    }
    const int64_t vi = (int64_t)b * a.n_pad + i;
    const float nu = a.vg[vi].x;
    const float bb = a.beta[b], th = a.theta[b];
    const float f = sigmoid_rate(a.Ucur[idx], bb, th);
    const float fp = a.q[i] * bb * f * (1.f - f);
    const float Wnu = a.A1 * s6[0] - a.A2 * s6[1];
    const float mu = -nu + fp * Wnu;
    float* cb = a.contrib + ((int64_t)b * 4) * a.n + i;
    cb[0] = nu * s6[2];
    cb[a.n] = nu * a.dA1c * s6[3];
    cb[2 * a.n] = -nu * s6[4];
    cb[3 * a.n] = -nu * a.dA2c * s6[5];
    const float bw[4] = {1.f / 6.f, 2.f / 6.f, 2.f / 6.f, 1.f / 6.f};
    const float cprev[4] = {0.f, 0.5f, 0.5f, 1.f};
    if (a.stg > 0) {
        const float accv = (a.stg == 3) ? mu : a.acc[idx] + mu;
        a.acc[idx] = accv;
        const float nun = a.dt * bw[a.stg - 1] * a.lam[idx] + cprev[a.stg] * a.dt * mu;
        a.vg[vi] = make_float2(nun, a.q[i] * sigmoid_rate(a.Uprev[idx], bb, th));
    } else {
        const float lamn = a.lam[idx] + (a.acc[idx] + mu);
        a.lam[idx] = lamn;
        if (a.Uprev)
            a.vg[vi] = make_float2(a.dt * bw[3] * lamn, a.q[i] * sigmoid_rate(a.Uprev[idx], bb, th));
    }
}

// gk[b][k] += sum_i contrib[b][k][i], one block per (b, k), fixed order
__global__ void adj_reduce_kernel(const float *__restrict__ contrib, int64_t n, double *__restrict__ gk) {
    __shared__ double red[256];
    const int64_t bk = blockIdx.x;
    const float *c = contrib + bk * n;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)c[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) gk[bk] += red[0];
}

__global__ void adj_finish_kernel(const double *__restrict__ gk, int cnt, float *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < cnt) out[t] = (float)gk[t];
}

SplitPlan mf_plan(nf_operator *op);

static SplitPlan adj_plan(nf_operator *op) {
    int res = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res, adj_pair_kernel, AD_THREADS, 0);
    return plan_splits(op->n_pad, AD_WARPS * AD_R, AD_TJ, std::max(res, 1));
}

}  // namespace nfi

using namespace nfi;

extern "C" nf_status nf_adjoint(nf_operator *op, const float *ckpt, int C, int B, double t0, double dt, int nsteps,
                                const float *beta, const float *theta, const nf_forcing *g, const float *lambda_T,
                                float *grad_u0, float *grad_kernel, void *stream) {
    clear_error();
    NF_ARG(op, "op is NULL");
    NF_ARG(ckpt && beta && theta && lambda_T && grad_u0 && grad_kernel, "array arguments must be non-NULL");
    NF_ARG(B >= 1 && B <= 65535 && C >= 1 && nsteps >= 0, "B, C or nsteps out of range");
    if (op->path != NF_MATRIX_FREE)
        return fail(NF_ERR_UNSUPPORTED, "nf_adjoint needs a matrix-free operator (W^T is applied on the fly)");
    if (g && g->kind != NF_FORCE_NONE && g->kind != NF_FORCE_MMS_EIGEN) return fail(NF_ERR_ARG, "unknown forcing");
    if (g && g->kind == NF_FORCE_MMS_EIGEN) NF_ARG(g->Y1 && g->Y2, "forcing: Y1 and Y2 are required");
    cudaStream_t s = as_stream(stream);
    const int64_t n = op->n, n_pad = op->n_pad;
    const size_t BN = (size_t)B * n;
    NF_TRY(ensure_workspace(op, B, mf_splits(op, B)));
    const SplitPlan apl = adj_plan(op);
    const int Cseg = std::min(C, std::max(nsteps, 1));
    float *stages = nullptr, *lam = nullptr, *acc = nullptr, *ubuf = nullptr, *part6 = nullptr, *contrib = nullptr;
    float2 *vg = nullptr;
    double *gk = nullptr;
    NF_CUDA_TRY(cudaMallocAsync(&stages, sizeof(float) * BN * 4 * Cseg, s));
    NF_CUDA_TRY(cudaMallocAsync(&lam, sizeof(float) * BN, s));
    NF_CUDA_TRY(cudaMallocAsync(&acc, sizeof(float) * BN, s));
    NF_CUDA_TRY(cudaMallocAsync(&ubuf, sizeof(float) * BN, s));
    NF_CUDA_TRY(cudaMallocAsync(&part6, sizeof(float) * 6 * apl.splits * (size_t)B * n_pad, s));
    NF_CUDA_TRY(cudaMallocAsync(&contrib, sizeof(float) * 4 * BN, s));
    NF_CUDA_TRY(cudaMallocAsync(&vg, sizeof(float2) * (size_t)B * n_pad, s));
    NF_CUDA_TRY(cudaMallocAsync(&gk, sizeof(double) * 4 * B, s));
    NF_CUDA_TRY(cudaMemsetAsync(vg, 0, sizeof(float2) * (size_t)B * n_pad, s));  // padded columns stay zero
    NF_CUDA_TRY(cudaMemsetAsync(gk, 0, sizeof(double) * 4 * B, s));
    NF_CUDA_TRY(cudaMemcpyAsync(lam, lambda_T, sizeof(float) * BN, cudaMemcpyDeviceToDevice, s));
    static const nf_forcing none{NF_FORCE_NONE, nullptr, nullptr, 0, 0, 0, 0, 0};
    const nf_forcing F = g ? *g : none;
    const nf_kernel &kp = op->kp;
    const float L2E = 1.4426950408889634f;
    const float c1 = -L2E / (kp.s1 * kp.s1), c2 = -L2E / (kp.s2 * kp.s2);
    const int T = 256;
    const unsigned eg = (unsigned)ceil_div((int64_t)BN, T);
    const int nseg = (nsteps + C - 1) / C;
    nf_status st = NF_OK;
    for (int seg = nseg - 1; seg >= 0 && st == NF_OK; --seg) {
        const int s0 = seg * C;
        const int cnt = std::min(C, nsteps - s0);
        // ---- recompute the segment forward, keeping every stage input
        NF_CUDA_TRY(cudaMemcpyAsync(ubuf, ckpt + (size_t)seg * BN, sizeof(float) * BN, cudaMemcpyDeviceToDevice, s));
        NF_TRY(launch_prep_g(op, ubuf, B, beta, theta, true, s));
        NF_TRY(launch_set_clock(op, t0 + (double)s0 * dt, s));
        for (int j = 0; j < cnt && st == NF_OK; ++j) {
            float *Sj = stages + (size_t)j * 4 * BN;
            NF_CUDA_TRY(cudaMemcpyAsync(Sj, ubuf, sizeof(float) * BN, cudaMemcpyDeviceToDevice, s));
            for (int stage = 1; stage <= 4; ++stage) {
                int splits = 1;
                NF_TRY(launch_mf_pair(op, B, s, &splits));
                StageParams p{};
                p.u = ubuf;
                p.beta = beta;
                p.theta = theta;
                p.forcing = F;
                p.dt = dt;
                p.stage = stage;
                p.ckpt = nullptr;
                p.C = 1;
                p.splits = splits;
                NF_TRY(launch_stage(op, B, p, s));
                if (stage < 4)
                    NF_CUDA_TRY(cudaMemcpyAsync(Sj + (size_t)stage * BN, op->U, sizeof(float) * BN,
                                                cudaMemcpyDeviceToDevice, s));
            }
        }
        // ---- reverse through the segment
        adj_prep_kernel<<<eg, T, 0, s>>>(lam, stages + ((size_t)(cnt - 1) * 4 + 3) * BN, op->q, beta, theta, n,
                                         n_pad, B, (float)(dt / 6.0), vg);
        NF_CUDA_TRY(cudaGetLastError());
        for (int j = cnt - 1; j >= 0; --j) {
            for (int stg = 3; stg >= 0; --stg) {
                dim3 grid((unsigned)apl.row_blocks, (unsigned)apl.splits);
                for (int b = 0; b < B; ++b)
                    adj_pair_kernel<<<grid, AD_THREADS, 0, s>>>(op->x4, vg, n_pad, B, b, apl.jchunk, c1, c2, part6,
                                                                op->err);
                AdjEpiArgs ea{};
                ea.partial = part6;
                ea.splits = apl.splits;
                ea.n = n;
                ea.n_pad = n_pad;
                ea.B = B;
                ea.stg = stg;
                ea.Ucur = stages + ((size_t)j * 4 + stg) * BN;
                ea.Uprev = (stg > 0) ? stages + ((size_t)j * 4 + stg - 1) * BN
                                     : (j > 0 ? stages + ((size_t)(j - 1) * 4 + 3) * BN : nullptr);
                ea.lam = lam;
                ea.acc = acc;
                ea.vg = vg;
                ea.contrib = contrib;
                ea.q = op->q;
                ea.beta = beta;
                ea.theta = theta;
                ea.A1 = kp.A1;
                ea.A2 = kp.A2;
                ea.dA1c = 2.f * kp.A1 / (kp.s1 * kp.s1 * kp.s1);
                ea.dA2c = 2.f * kp.A2 / (kp.s2 * kp.s2 * kp.s2);
                ea.dt = (float)dt;
                adj_epilogue_kernel<<<eg, T, 0, s>>>(ea);
                adj_reduce_kernel<<<(unsigned)(4 * B), 256, 0, s>>>(contrib, n, gk);
                NF_CUDA_TRY(cudaGetLastError());
            }
        }
    }
    NF_CUDA_TRY(cudaMemcpyAsync(grad_u0, lam, sizeof(float) * BN, cudaMemcpyDeviceToDevice, s));
    adj_finish_kernel<<<(unsigned)ceil_div(4 * B, 256), 256, 0, s>>>(gk, 4 * B, grad_kernel);
    NF_CUDA_TRY(cudaGetLastError());
    cudaFreeAsync(stages, s);
    cudaFreeAsync(lam, s);
    cudaFreeAsync(acc, s);
    cudaFreeAsync(ubuf, s);
    cudaFreeAsync(part6, s);
    cudaFreeAsync(contrib, s);
    cudaFreeAsync(vg, s);
    cudaFreeAsync(gk, s);
    return st;
}
