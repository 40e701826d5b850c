// nf_models.cu -- the §5 models on any single operator path: the neural field of Eq. (2.9)
// or the synaptic-depression model of Eq. (nfsyndep),
//     du/dt = -u + sum_j w_ij mu_j s_j f(u_j),     tau ds/dt = 1 - s - beta_d s f(u),
// with the sigmoid firing rate or the C^4 smooth step of Eq. (smoothf), advanced by the
// classical RK4 tableau or by Adams-Bashforth 5 (one nonlocal sum per step).  AB5 is
// started by four RK4 steps whose first-stage derivatives seed its history.
//
// The nonlocal sums are the operator's own kernels (matrix-free, dense FP32, bf16 hi+lo,
// symmetric dense) on g = mu o s o f(u) (mu folded into the dense W diag(q) paths); the
// kernels here are elementwise: the g preparation, a fused two-field RK4 stage and a
// fused AB5 step, each reducing the operator's partial-sum slots in a fixed order.
#include "nf_internal.cuh"

namespace nfi {

struct ModelArgs {
    int kind;              // NF_MODEL_FIELD or NF_MODEL_DEPRESSION
    int rate;              // NF_RATE_SIGMOID or NF_RATE_SMOOTHSTEP
    float a, inv_ba;       // smooth step: lower end and 1 / (b - a)
    float b;
    float tau_inv, beta_d;
};

// Firing rate.  Smooth step: with t = (u - a)/(b - a) in [0, 1], the degree-9 polynomial
// t^5 (126 - 420 t + 540 t^2 - 315 t^3 + 70 t^4), the one with value 0 and four zero
// derivatives at t = 0 and value 1 and four zero derivatives at t = 1.
__device__ __forceinline__ float model_rate(const ModelArgs &m, float u, float beta, float theta) {
    if (m.rate == NF_RATE_SMOOTHSTEP) {
        if (u < m.a) return 0.f;
        if (u >= m.b) return 1.f;
        const float t = (u - m.a) * m.inv_ba;
        const float p = fmaf(fmaf(fmaf(fmaf(70.f, t, -315.f), t, 540.f), t, -420.f), t, 126.f);
        const float t2 = t * t;
        return t2 * t2 * t * p;
    }
    return 1.0f / (1.0f + expf(-beta * (u - theta)));
}

struct ModelState {
    float *u, *s;            // caller's state (s: depression only)
    float *U, *S;            // current stage inputs
    float *ku, *ksd;         // RK4 slope accumulators (u, s)
    float *hu, *hs;          // AB5 history: 5 slots of B x n each (u, s)
    float *g;                // [B][n_pad] input of the nonlocal sum
    const float *q;          // mu, or null when folded into W
    const float *rs;         // bf16 hi+lo row scales, or null
    const float *partial;
    int splits;
    int64_t n, n_pad;
    int B;
    const float *beta, *theta;
};

__device__ __forceinline__ void write_g(const ModelState &st, const ModelArgs &m, int b, int64_t i, int64_t idx,
                                        float u, float s) {
    const float f = model_rate(m, u, st.beta[b], st.theta[b]);
    float gv = (m.kind == NF_MODEL_DEPRESSION) ? s * f : f;
    if (st.q) gv *= st.q[i];
    st.g[(int64_t)b * st.n_pad + i] = gv;
}

__device__ __forceinline__ float slot_sum(const ModelState &st, int b, int64_t i) {
    float I = 0.f;
    for (int sp = 0; sp < st.splits; ++sp) I += st.partial[((int64_t)sp * st.B + b) * st.n_pad + i];
    return st.rs ? I * st.rs[i] : I;
}

// g from (u, s); U = u, S = s
__global__ void model_prep_kernel(ModelState st, ModelArgs m) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)st.B * st.n) return;
    const int b = (int)(idx / st.n);
    const int64_t i = idx - (int64_t)b * st.n;
    const float u = st.u[idx];
    const float s = (m.kind == NF_MODEL_DEPRESSION) ? st.s[idx] : 1.f;
    st.U[idx] = u;
    if (m.kind == NF_MODEL_DEPRESSION) st.S[idx] = s;
    write_g(st, m, b, i, idx, u, s);
}

// RK4 stage `stage` (1..4) of both fields; hist >= 0: store the stage-1 derivative in AB5
// history slot hist.  Writes the next stage's inputs and their g.
__global__ void model_rk4_stage_kernel(ModelState st, ModelArgs m, int stage, float dt, int hist) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)st.B * st.n) return;
    const int b = (int)(idx / st.n);
    const int64_t i = idx - (int64_t)b * st.n;
    const bool dep = m.kind == NF_MODEL_DEPRESSION;
    const float Uv = st.U[idx], Sv = dep ? st.S[idx] : 1.f;
    const float ku = -Uv + slot_sum(st, b, i);
    const float ks = dep ? (1.f - Sv - m.beta_d * Sv * model_rate(m, Uv, st.beta[b], st.theta[b])) * m.tau_inv : 0.f;
    if (hist >= 0) {
        const int64_t h = (int64_t)hist * st.B * st.n + idx;
        st.hu[h] = ku;
        if (dep) st.hs[h] = ks;
    }
    float Un, Sn = 1.f;
    const float uv = st.u[idx], sv = dep ? st.s[idx] : 1.f;
    if (stage == 1) {
        st.ku[idx] = ku;
        Un = fmaf(0.5f * dt, ku, uv);
        if (dep) {
            st.ksd[idx] = ks;
            Sn = fmaf(0.5f * dt, ks, sv);
        }
    } else if (stage == 2 || stage == 3) {
        const float c = (stage == 2) ? 0.5f * dt : dt;
        st.ku[idx] = fmaf(2.f, ku, st.ku[idx]);
        Un = fmaf(c, ku, uv);
        if (dep) {
            st.ksd[idx] = fmaf(2.f, ks, st.ksd[idx]);
            Sn = fmaf(c, ks, sv);
        }
    } else {
        Un = fmaf(dt / 6.f, st.ku[idx] + ku, uv);
        st.u[idx] = Un;
        if (dep) {
            Sn = fmaf(dt / 6.f, st.ksd[idx] + ks, sv);
            st.s[idx] = Sn;
        }
    }
    st.U[idx] = Un;
    if (dep) st.S[idx] = Sn;
    write_g(st, m, b, i, idx, Un, Sn);
}

// Adams-Bashforth 5 step `step` (>= 4): F_step into history slot step % 5, then
// y += dt (1901 F_n - 2774 F_{n-1} + 2616 F_{n-2} - 1274 F_{n-3} + 251 F_{n-4}) / 720.
__global__ void model_ab5_kernel(ModelState st, ModelArgs m, int step, float dt) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)st.B * st.n) return;
    const int b = (int)(idx / st.n);
    const int64_t i = idx - (int64_t)b * st.n;
    const bool dep = m.kind == NF_MODEL_DEPRESSION;
    const int64_t plane = (int64_t)st.B * st.n;
    const float uv = st.u[idx], sv = dep ? st.s[idx] : 1.f;
    const float Fu = -uv + slot_sum(st, b, i);
    const float Fs = dep ? (1.f - sv - m.beta_d * sv * model_rate(m, uv, st.beta[b], st.theta[b])) * m.tau_inv : 0.f;
    st.hu[(int64_t)(step % 5) * plane + idx] = Fu;
    if (dep) st.hs[(int64_t)(step % 5) * plane + idx] = Fs;
    const float c[5] = {1901.f / 720.f, -2774.f / 720.f, 2616.f / 720.f, -1274.f / 720.f, 251.f / 720.f};
    float du = 0.f, ds = 0.f;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int64_t h = (int64_t)((step - k) % 5) * plane + idx;
        du = fmaf(c[k], st.hu[h], du);
        if (dep) ds = fmaf(c[k], st.hs[h], ds);
    }
    const float un = fmaf(dt, du, uv);
    st.u[idx] = un;
    float sn = 1.f;
    if (dep) {
        sn = fmaf(dt, ds, sv);
        st.s[idx] = sn;
    }
    write_g(st, m, b, i, idx, un, sn);
}

}  // namespace nfi

using namespace nfi;

extern "C" nf_status nf_field_advance(nf_operator *op, const nf_model *model, int integrator, float *u, float *s,
                                      int B, double dt, int nsteps, const float *beta, const float *theta,
                                      void *stream) {
    clear_error();
    NF_ARG(op && model && u && beta && theta, "op, model, u, beta and theta must be non-NULL");
    NF_ARG(op->path != NF_GROUPED, "nf_field_advance takes a single-operator path (not a grouped operator)");
    NF_ARG(model->kind == NF_MODEL_FIELD || model->kind == NF_MODEL_DEPRESSION, "unknown model kind %d", model->kind);
    NF_ARG(model->rate == NF_RATE_SIGMOID || model->rate == NF_RATE_SMOOTHSTEP, "unknown firing rate %d", model->rate);
    NF_ARG(integrator == NF_INTEGRATOR_RK4 || integrator == NF_INTEGRATOR_AB5, "unknown integrator %d", integrator);
    NF_ARG(model->kind != NF_MODEL_DEPRESSION || s, "the depression model needs the efficacy field s");
    NF_ARG(model->rate != NF_RATE_SMOOTHSTEP || model->b > model->a, "smooth step needs b > a");
    NF_ARG(model->kind != NF_MODEL_DEPRESSION || model->tau > 0.f, "the depression model needs tau > 0");
    NF_ARG(B >= 1 && B <= 65535 && nsteps >= 0 && dt > 0.0, "B, nsteps or dt out of range");
    cudaStream_t cs = as_stream(stream);
    const bool dep = model->kind == NF_MODEL_DEPRESSION;
    const bool ab5 = integrator == NF_INTEGRATOR_AB5;
    const int64_t BN = (int64_t)B * op->n;
    NF_TRY(ensure_workspace(op, B, nonlocal_splits(op, B)));
    float *extra = nullptr;  // S, ksd (depression), AB5 history u (and s)
    const int64_t nextra = (dep ? 2 : 0) * BN + (ab5 ? (dep ? 10 : 5) * BN : 0);
    if (nextra > 0) NF_CUDA_TRY(cudaMallocAsync(&extra, sizeof(float) * nextra, cs));
    ModelState st{};
    st.u = u;
    st.s = dep ? s : nullptr;
    st.U = op->U;
    st.ku = op->ks;
    float *p = extra;
    if (dep) {
        st.S = p, p += BN;
        st.ksd = p, p += BN;
    }
    if (ab5) {
        st.hu = p, p += 5 * BN;
        if (dep) st.hs = p, p += 5 * BN;
    }
    st.g = op->g;
    st.q = q_on_vector(op) ? op->q : nullptr;
    st.rs = (op->path == NF_DENSE_BF16X2) ? op->rs : nullptr;
    st.partial = op->partial;
    st.n = op->n;
    st.n_pad = op->n_pad;
    st.B = B;
    st.beta = beta;
    st.theta = theta;
    ModelArgs m{};
    m.kind = model->kind;
    m.rate = model->rate;
    m.a = model->a;
    m.b = model->b;
    m.inv_ba = model->rate == NF_RATE_SMOOTHSTEP ? 1.f / (model->b - model->a) : 0.f;
    m.tau_inv = dep ? 1.f / model->tau : 0.f;
    m.beta_d = model->beta_d;
    const int T = 256;
    const unsigned grid = (unsigned)ceil_div(BN, T);
    const float dtf = (float)dt;
    nf_status status = NF_OK;
    auto run = [&]() -> nf_status {
        model_prep_kernel<<<grid, T, 0, cs>>>(st, m);
        NF_CUDA_TRY(cudaGetLastError());
        for (int step = 0; step < nsteps; ++step) {
            if (ab5 && step >= 4) {
                int splits = 1;
                NF_TRY(launch_nonlocal_partial(op, B, cs, &splits));
                st.splits = splits;
                model_ab5_kernel<<<grid, T, 0, cs>>>(st, m, step, dtf);
                NF_CUDA_TRY(cudaGetLastError());
                continue;
            }
            for (int stage = 1; stage <= 4; ++stage) {
                int splits = 1;
                NF_TRY(launch_nonlocal_partial(op, B, cs, &splits));
                st.splits = splits;
                model_rk4_stage_kernel<<<grid, T, 0, cs>>>(st, m, stage, dtf, (ab5 && stage == 1) ? step : -1);
                NF_CUDA_TRY(cudaGetLastError());
            }
        }
        return NF_OK;
    };
    status = run();
    if (extra) cudaFreeAsync(extra, cs);
    return status;
}
