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
// The adjoint pair kernel (adj_sym_kernel, with the forward symmetric kernel's block-pair
// schedule: each unordered pair evaluated once) computes W nu as partial-slot sums and the
// four parameter sums sum_ij nu_i g_j (e1, r^2 e1, e2, r^2 e2) as per-CTA partials.  The
// epilogue adds the slots, applies the recurrences and prepares (nu, g) of the next stage;
// a fixed-order FP64 reduction accumulates the parameter gradients.  Stage inputs are
// recomputed segment by segment from checkpoints, on a second stream: while segment k is
// reversed on the caller's stream, segment k - 1 is recomputed into the other of two stage
// buffers, so each launch's last, partly filled wave and the small elementwise kernels of
// one stream overlap the other's pair kernels.  The results do not depend on the overlap
// (every kernel's summation order is fixed).
#include "nf_internal.cuh"

#include <algorithm>

namespace nfi {

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
    const float *wpart;      // [slots][B][n_pad]: partial sums of W nu
    int slots;
    int64_t n, n_pad;
    int B;
    int stg;                 // 0..3 (stage s = stg + 1)
    const float *Ucur;       // U_s
    const float *Uprev;      // U_{s-1} (stg > 0), U_4 of the previous step (stg == 0), or null
    float *lam, *acc;
    float2 *vg;
    const float *q, *beta, *theta;
    float dt;
};

__global__ void adj_epilogue_kernel(AdjEpiArgs a) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)a.B * a.n) return;
    const int b = (int)(idx / a.n);
    const int64_t i = idx - (int64_t)b * a.n;
    const float Wnu = sum_slots(a.wpart + (int64_t)b * a.n_pad + i, (int64_t)a.B * a.n_pad, a.slots);
    const int64_t vi = (int64_t)b * a.n_pad + i;
    const float nu = a.vg[vi].x;
    const float bb = a.beta[b], th = a.theta[b];
    const float f = sigmoid_rate(a.Ucur[idx], bb, th);
    const float fp = a.q[i] * bb * f * (1.f - f);
    const float mu = -nu + fp * Wnu;
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

// gk[b][k] += scale[k] * sum_c gpart[b][c][k] over the CTAs c of the stage's pair launch,
// one block per (b, k), fixed order.  scale = (1, 2 A1 / s1^3 * r2phys, -1, -2 A2 / s2^3 *
// r2phys): d w / dA1 = e1, d w / ds1 = 2 A1 r^2 e1 / s1^3, d w / dA2 = -e2,
// d w / ds2 = -2 A2 r^2 e2 / s2^3, with r^2 converted from exponent units.
struct AdjScale {
    double k[4];
};
__global__ void adj_reduce_kernel(const float *__restrict__ gpart, int64_t ncta, AdjScale sc, double *__restrict__ gk) {
    __shared__ double red[256];
    const int b = blockIdx.x >> 2, k = blockIdx.x & 3;
    const float *c = gpart + (int64_t)b * ncta * 4 + k;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < ncta; i += blockDim.x) s += (double)c[i * 4];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) gk[blockIdx.x] += sc.k[k] * red[0];
}

__global__ void adj_finish_kernel(const double *__restrict__ gk, int cnt, float *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < cnt) out[t] = (float)gk[t];
}

// Stream-ordered scratch buffers of one call, released on every return path (an early
// return after a failed launch or allocation frees what was allocated before it).
struct StreamScratch {
    cudaStream_t s;
    void *p[8] = {};
    int count = 0;
    explicit StreamScratch(cudaStream_t st) : s(st) {}
    StreamScratch(const StreamScratch &) = delete;
    StreamScratch &operator=(const StreamScratch &) = delete;
    template <typename T>
    cudaError_t alloc(T **out, size_t bytes) {
        *out = nullptr;
        if (count == 8) return cudaErrorInvalidValue;
        void *q = nullptr;
        const cudaError_t e = cudaMallocAsync(&q, bytes, s);
        if (e != cudaSuccess) return e;
        p[count++] = q;
        *out = static_cast<T *>(q);
        return cudaSuccess;
    }
    ~StreamScratch() {
        for (int i = 0; i < count; ++i) cudaFreeAsync(p[i], s);
    }
};

// A second stream forked from the caller's, on which checkpoint segments are recomputed
// while the previous segment is reversed on the caller's stream.  Events: fork, join, and per
// stage buffer "recomputed" and "reversed".  The destructor joins the side stream back into
// the caller's stream (on every return path, before the scratch buffers are released), so
// the call stays stream-ordered on the caller's stream as a whole.
struct SideStream {
    cudaStream_t main, side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, rec[2] = {}, rev[2] = {};
    bool forked = false;
    explicit SideStream(cudaStream_t m) : main(m) {}
    SideStream(const SideStream &) = delete;
    SideStream &operator=(const SideStream &) = delete;
    cudaError_t start() {
        cudaError_t e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
        cudaEvent_t *evs[6] = {&fork, &join, &rec[0], &rec[1], &rev[0], &rev[1]};
        for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(evs[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(fork, main);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side, fork, 0);
        forked = e == cudaSuccess;
        return e;
    }
    ~SideStream() {
        if (forked && cudaEventRecord(join, side) == cudaSuccess) cudaStreamWaitEvent(main, join, 0);
        cudaEvent_t evs[6] = {fork, join, rec[0], rec[1], rev[0], rev[1]};
        for (cudaEvent_t ev : evs)
            if (ev) cudaEventDestroy(ev);
        if (side) cudaStreamDestroy(side);
    }
};

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
    if (g && (g->kind == NF_FORCE_MMS_FLAT || g->kind == NF_FORCE_MMS_SPHERE))
        return fail(NF_ERR_UNSUPPORTED, "this manufactured forcing depends on the kernel parameters; nf_adjoint "
                                        "treats forcing as data and does not differentiate it");
    if (g && g->kind != NF_FORCE_NONE && g->kind != NF_FORCE_MMS_EIGEN) return fail(NF_ERR_ARG, "unknown forcing");
    if (g && g->kind == NF_FORCE_MMS_EIGEN) NF_ARG(g->Y1 && g->Y2, "forcing: Y1 and Y2 are required");
    cudaStream_t s = as_stream(stream);
    const int64_t n = op->n, n_pad = op->n_pad;
    const size_t BN = (size_t)B * n;
    NF_TRY(ensure_workspace(op, B, mf_splits(op, B)));
    // block-pair culling (nf_operator_mf_cull): the adjoint kernel runs over its own live
    // pairs, and each node's live W nu slots are added into slot 0 before the epilogue
    const bool cull = op->mf_cull && op->adj_pairs;
    const int Cseg = std::min(C, std::max(nsteps, 1));
    float *stages = nullptr, *lam = nullptr, *acc = nullptr, *ubuf = nullptr, *wpart = nullptr, *gpart = nullptr;
    float2 *vg = nullptr;
    double *gk = nullptr;
    StreamScratch scratch(s);  // freed (stream-ordered) on every return below
    // two stage buffers: segment k - 1 is recomputed into one while segment k is reversed
    // from the other
    const size_t seg_elems = BN * 4 * (size_t)Cseg;
    NF_CUDA_TRY(scratch.alloc(&stages, sizeof(float) * 2 * seg_elems));
    NF_CUDA_TRY(scratch.alloc(&lam, sizeof(float) * BN));
    NF_CUDA_TRY(scratch.alloc(&acc, sizeof(float) * BN));
    NF_CUDA_TRY(scratch.alloc(&ubuf, sizeof(float) * BN));
    // W nu slots and parameter partials for the smallest node block the kernel may take
    NF_CUDA_TRY(scratch.alloc(&wpart, sizeof(float) * (size_t)adj_slot_capacity(op) * B * n_pad));
    NF_CUDA_TRY(scratch.alloc(&gpart, sizeof(float) * 4 * (size_t)B * adj_pair_capacity(op)));
    NF_CUDA_TRY(scratch.alloc(&vg, sizeof(float2) * (size_t)B * n_pad));
    NF_CUDA_TRY(scratch.alloc(&gk, sizeof(double) * 4 * B));
    NF_CUDA_TRY(cudaMemsetAsync(vg, 0, sizeof(float2) * (size_t)B * n_pad, s));  // padded columns stay zero
    NF_TRY(adj_autotune(op, vg, B, wpart, gpart, s));  // first call on this operator only
    const int slots = adj_slots(op);  // one W nu slot per node block of the chosen shape
    const int64_t ncta = sym_pair_count(op);
    const int64_t ncta_run = cull ? op->adj_live : ncta;
    NF_CUDA_TRY(cudaMemsetAsync(gk, 0, sizeof(double) * 4 * B, s));
    NF_CUDA_TRY(cudaMemcpyAsync(lam, lambda_T, sizeof(float) * BN, cudaMemcpyDeviceToDevice, s));
    static const nf_forcing none{NF_FORCE_NONE, nullptr, nullptr, 0, 0, 0, 0, 0, 0, 0, 0};
    const nf_forcing F = g ? *g : none;
    const nf_kernel &kp = op->kp;
    const int T = 256;
    const unsigned eg = (unsigned)ceil_div((int64_t)BN, T);
    const int nseg = (nsteps + C - 1) / C;
    // ---- recompute segment seg forward into st, keeping every stage input (stream ss)
    auto recompute = [&](int seg, float *st, cudaStream_t ss) -> nf_status {
        const int s0 = seg * C;
        const int cnt = std::min(C, nsteps - s0);
        NF_CUDA_TRY(cudaMemcpyAsync(ubuf, ckpt + (size_t)seg * BN, sizeof(float) * BN, cudaMemcpyDeviceToDevice, ss));
        NF_TRY(launch_prep_g(op, ubuf, B, beta, theta, true, ss));
        NF_TRY(launch_set_clock(op, t0 + (double)s0 * dt, ss));
        for (int j = 0; j < cnt; ++j) {
            float *Sj = st + (size_t)j * 4 * BN;
            NF_CUDA_TRY(cudaMemcpyAsync(Sj, ubuf, sizeof(float) * BN, cudaMemcpyDeviceToDevice, ss));
            for (int stage = 1; stage <= 4; ++stage) {
                int splits = 1;
                NF_TRY(launch_mf_pair(op, B, ss, &splits));
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
                NF_TRY(launch_stage(op, B, p, ss));
                if (stage < 4)
                    NF_CUDA_TRY(cudaMemcpyAsync(Sj + (size_t)stage * BN, op->U, sizeof(float) * BN,
                                                cudaMemcpyDeviceToDevice, ss));
            }
        }
        return NF_OK;
    };
    SideStream side(s);  // joined into s before the scratch buffers are released
    if (nseg > 0) {
        NF_CUDA_TRY(side.start());
        NF_TRY(recompute(nseg - 1, stages + (size_t)((nseg - 1) & 1) * seg_elems, side.side));
        NF_CUDA_TRY(cudaEventRecord(side.rec[(nseg - 1) & 1], side.side));
    }
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int cnt = std::min(C, nsteps - seg * C);
        const int bufi = seg & 1;
        // the next segment back is recomputed on the side stream while this one is reversed;
        // its buffer was last read by the reverse pass of segment seg + 1
        if (seg >= 1) {
            if (seg + 1 < nseg) NF_CUDA_TRY(cudaStreamWaitEvent(side.side, side.rev[(seg + 1) & 1], 0));
            NF_TRY(recompute(seg - 1, stages + (size_t)((seg - 1) & 1) * seg_elems, side.side));
            NF_CUDA_TRY(cudaEventRecord(side.rec[(seg - 1) & 1], side.side));
        }
        NF_CUDA_TRY(cudaStreamWaitEvent(s, side.rec[bufi], 0));
        float *const segst = stages + (size_t)bufi * seg_elems;
        // ---- reverse through the segment
        adj_prep_kernel<<<eg, T, 0, s>>>(lam, segst + ((size_t)(cnt - 1) * 4 + 3) * BN, op->q, beta, theta, n,
                                         n_pad, B, (float)(dt / 6.0), vg);
        NF_CUDA_TRY(cudaGetLastError());
        for (int j = cnt - 1; j >= 0; --j) {
            for (int stg = 3; stg >= 0; --stg) {
                float r2phys = 1.f;
                for (int b = 0; b < B; ++b) {
                    NF_TRY(launch_adj_sym(op, vg, B, b, wpart, gpart, &r2phys, s));
                    if (cull) NF_TRY(launch_adj_cull_reduce(op, wpart, B, b, s));
                }
                AdjEpiArgs ea{};
                ea.wpart = wpart;
                ea.slots = cull ? 1 : slots;
                ea.n = n;
                ea.n_pad = n_pad;
                ea.B = B;
                ea.stg = stg;
                ea.Ucur = segst + ((size_t)j * 4 + stg) * BN;
                ea.Uprev = (stg > 0) ? segst + ((size_t)j * 4 + stg - 1) * BN
                                     : (j > 0 ? segst + ((size_t)(j - 1) * 4 + 3) * BN : nullptr);
                ea.lam = lam;
                ea.acc = acc;
                ea.vg = vg;
                ea.q = op->q;
                ea.beta = beta;
                ea.theta = theta;
                ea.dt = (float)dt;
                AdjScale sc{{1.0, 2.0 * kp.A1 / ((double)kp.s1 * kp.s1 * kp.s1) * r2phys, -1.0,
                             -2.0 * kp.A2 / ((double)kp.s2 * kp.s2 * kp.s2) * r2phys}};
                adj_reduce_kernel<<<(unsigned)(4 * B), 256, 0, s>>>(gpart, ncta_run, sc, gk);
                adj_epilogue_kernel<<<eg, T, 0, s>>>(ea);
                NF_CUDA_TRY(cudaGetLastError());
            }
        }
        NF_CUDA_TRY(cudaEventRecord(side.rev[bufi], s));  // segst may now be overwritten
    }
    NF_CUDA_TRY(cudaMemcpyAsync(grad_u0, lam, sizeof(float) * BN, cudaMemcpyDeviceToDevice, s));
    adj_finish_kernel<<<(unsigned)ceil_div(4 * B, 256), 256, 0, s>>>(gk, 4 * B, grad_kernel);
    NF_CUDA_TRY(cudaGetLastError());
    return NF_OK;
}
