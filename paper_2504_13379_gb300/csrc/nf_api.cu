// nf_api.cu -- C ABI entry points: errors, operator lifecycle, nonlocal apply and the
// graph-captured RK4 driver.
#include "nf_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

namespace nfi {

static thread_local char g_err[1024] = "";

nf_status fail(nf_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

nf_status cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    const char *base = strrchr(file, '/');
    snprintf(g_err, sizeof(g_err), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), base ? base + 1 : file,
             line);
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? NF_ERR_NOMEM : NF_ERR_CUDA;
}

void clear_error() { g_err[0] = 0; }

int device_id() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

int num_sms() {
    static int cached[64] = {0};
    const int d = device_id();
    if (d >= 0 && d < 64 && cached[d]) return cached[d];
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
    if (v <= 0) v = 1;
    if (d >= 0 && d < 64) cached[d] = v;
    return v;
}

// ---------------------------------------------------------------- workspace
nf_status ensure_workspace(nf_operator *op, int B, int splits) {
    const size_t need_p = (size_t)splits * B * op->n_pad;
    const size_t need_g = (size_t)B * op->n_pad;
    const size_t need_s = (size_t)B * op->n;
    // captured graphs hold workspace pointers: drop them before anything moves
    if (need_p > op->partial_cap || need_g > op->g_cap || need_s > op->state_cap) destroy_graphs(op);
    if (need_p > op->partial_cap) {
        if (op->partial) NF_CUDA_TRY(cudaFree(op->partial));
        op->partial = nullptr;
        op->partial_cap = 0;
        NF_CUDA_TRY(cudaMalloc(&op->partial, need_p * sizeof(float)));
        op->partial_cap = need_p;
    }
    if (need_g > op->g_cap) {
        if (op->g) NF_CUDA_TRY(cudaFree(op->g));
        op->g = nullptr;
        op->g_cap = 0;
        NF_CUDA_TRY(cudaMalloc(&op->g, need_g * sizeof(float)));
        NF_CUDA_TRY(cudaMemset(op->g, 0, need_g * sizeof(float)));  // padding columns stay zero
        op->g_cap = need_g;
    }
    if (need_s > op->state_cap) {
        if (op->U) NF_CUDA_TRY(cudaFree(op->U));
        if (op->ks) NF_CUDA_TRY(cudaFree(op->ks));
        op->U = op->ks = nullptr;
        op->state_cap = 0;
        NF_CUDA_TRY(cudaMalloc(&op->U, need_s * sizeof(float)));
        NF_CUDA_TRY(cudaMalloc(&op->ks, need_s * sizeof(float)));
        op->state_cap = need_s;
    }
    return NF_OK;
}

SplitPlan mf_plan(nf_operator *op);
SplitPlan dense_plan(nf_operator *op);

int nonlocal_splits(nf_operator *op, int B) {
    return (op->path == NF_MATRIX_FREE) ? mf_splits(op, B) : dense_splits(op, B);
}

nf_status launch_nonlocal_partial(nf_operator *op, int B, cudaStream_t s, int *splits_out) {
    if (op->path == NF_MATRIX_FREE) return launch_mf_pair(op, B, s, splits_out);
    return launch_dense_gemv(op, B, s, splits_out);
}

// ---------------------------------------------------------------- pack kernel
// x4: coordinates as float4; xyz: coordinates times `scale` (= sqrt(log2 e) / s1) as
// structure of arrays, so squared scaled distances are exponents of 2 for the SFU.
__global__ void pack_nodes_kernel(const float *__restrict__ x, const float *__restrict__ q, int64_t n,
                                  int64_t n_pad, float scale, float4 *__restrict__ x4, float *__restrict__ xyz,
                                  float *__restrict__ qp) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_pad) return;
    const bool in = j < n;
    const float a = in ? x[3 * j] : 0.f, b = in ? x[3 * j + 1] : 0.f, c = in ? x[3 * j + 2] : 0.f;
    x4[j] = make_float4(a, b, c, 0.f);
    xyz[j] = a * scale;
    xyz[n_pad + j] = b * scale;
    xyz[2 * n_pad + j] = c * scale;
    qp[j] = in ? q[j] : 0.f;
}

// Failure-path self-test: waits on an mbarrier whose phase nothing completes, with a
// small poll limit; the wait gives up and records a timeout instead of hanging.
__global__ void selftest_wait_kernel(int *flag, long long polls) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    bool done = false;
    for (long long i = 0; i < polls && !done; ++i) done = mbar_try_wait(&bar, 0);
    if (!done && threadIdx.x == 0) set_dev_error(flag, DEV_TIMEOUT);
}

// ---------------------------------------------------------------- graph cache
}  // namespace nfi

struct nf_graph_cache {
    bool valid = false;
    float *u = nullptr;
    int B = 0;
    const float *beta = nullptr, *theta = nullptr;
    nf_forcing F{};
    double dt = 0;
    bool profile = false;
    float *ckpt = nullptr;
    int C = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphNode_t prof_nodes[8] = {};  // the graph's event-record nodes, by event index
};

namespace nfi {

void destroy_graphs(nf_operator *op) {
    if (!op->graphs) return;
    nf_graph_cache *c = op->graphs;
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
    op->graphs = nullptr;
}

static bool same_forcing(const nf_forcing &a, const nf_forcing &b) {
    return a.kind == b.kind && a.Y1 == b.Y1 && a.Y2 == b.Y2 && a.c == b.c && a.a0 == b.a0 && a.lam0 == b.lam0 &&
           a.lam1 == b.lam1 && a.lam2 == b.lam2 && a.radius == b.radius && a.sigma == b.sigma && a.scale == b.scale;
}

// One RK4 step = 4 x (nonlocal partial sums, fused stage kernel), captured once.
static nf_status rk4_step_graph(nf_operator *op, float *u, int B, double dt, const float *beta,
                                const float *theta, const nf_forcing &F, float *ckpt, int C, cudaGraphExec_t *out) {
    if (!op->graphs) op->graphs = new nf_graph_cache();
    nf_graph_cache *c = op->graphs;
    if (c->valid && c->u == u && c->B == B && c->beta == beta && c->theta == theta && same_forcing(c->F, F) &&
        c->dt == dt && c->ckpt == ckpt && c->C == C && c->profile == op->profile) {
        *out = c->exec;
        return NF_OK;
    }
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->exec = nullptr;
    c->graph = nullptr;
    c->valid = false;
    if (!c->cap_stream) NF_CUDA_TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = c->cap_stream;
    NF_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    nf_status st = NF_OK;
    for (int stage = 1; stage <= 4 && st == NF_OK; ++stage) {
        int splits = 1;
        if (op->profile) {
            cudaError_t pe = cudaEventRecordWithFlags(op->prof_ring[2 * (stage - 1)], cs, cudaEventRecordExternal);
            if (pe != cudaSuccess) {
                st = cuda_fail(pe, "cudaEventRecord", __FILE__, __LINE__);
                break;
            }
        }
        if (op->path == NF_GROUPED) {
            // stage s reads the F buffer written by stage s-1: odd stages read buffer 0
            st = tc_launch(op, (stage - 1) & 1, 1, nullptr, u, beta, theta, dt, stage, ckpt, C, cs);
            if (st == NF_OK && op->profile) {
                cudaError_t pe = cudaEventRecordWithFlags(op->prof_ring[2 * (stage - 1) + 1], cs, cudaEventRecordExternal);
                if (pe != cudaSuccess) st = cuda_fail(pe, "cudaEventRecord", __FILE__, __LINE__);
            }
            continue;
        }
        st = launch_nonlocal_partial(op, B, cs, &splits);
        if (st != NF_OK) break;
        if (op->profile) {
            cudaError_t pe = cudaEventRecordWithFlags(op->prof_ring[2 * (stage - 1) + 1], cs, cudaEventRecordExternal);
            if (pe != cudaSuccess) {
                st = cuda_fail(pe, "cudaEventRecord", __FILE__, __LINE__);
                break;
            }
        }
        StageParams p{};
        p.u = u;
        p.beta = beta;
        p.theta = theta;
        p.forcing = F;
        p.dt = dt;
        p.stage = stage;
        p.ckpt = ckpt;
        p.C = C;
        p.splits = splits;
        st = launch_stage(op, B, p, cs);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (st != NF_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    e = cudaGraphInstantiate(&c->exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
    }
    c->graph = g;
    if (op->profile) {  // find the event-record nodes, so replays can retarget them
        size_t cnt = 0;
        NF_CUDA_TRY(cudaGraphGetNodes(g, nullptr, &cnt));
        cudaGraphNode_t *nodes = new cudaGraphNode_t[cnt];
        cudaError_t ge = cudaGraphGetNodes(g, nodes, &cnt);
        for (int k = 0; k < 8; ++k) c->prof_nodes[k] = nullptr;
        for (size_t i = 0; i < cnt && ge == cudaSuccess; ++i) {
            cudaGraphNodeType ty;
            ge = cudaGraphNodeGetType(nodes[i], &ty);
            if (ge != cudaSuccess || ty != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev = nullptr;
            ge = cudaGraphEventRecordNodeGetEvent(nodes[i], &ev);
            for (int k = 0; k < 8 && ge == cudaSuccess; ++k)
                if (ev == op->prof_ring[k]) c->prof_nodes[k] = nodes[i];
        }
        delete[] nodes;
        if (ge != cudaSuccess) return cuda_fail(ge, "cudaGraphGetNodes (profiling events)", __FILE__, __LINE__);
        for (int k = 0; k < 8; ++k)
            if (!c->prof_nodes[k]) return fail(NF_ERR_CUDA, "profiling event %d not found in the step graph", k);
    }
    c->valid = true;
    c->u = u;
    c->B = B;
    c->beta = beta;
    c->theta = theta;
    c->F = F;
    c->dt = dt;
    c->profile = op->profile;
    c->ckpt = ckpt;
    c->C = C;
    *out = c->exec;
    return NF_OK;
}

// Replay the captured step nsteps times; with profiling on, each replay records its stage
// timings into the next slot of the operator's event ring.
static nf_status launch_steps(nf_operator *op, cudaGraphExec_t exec, int nsteps, cudaStream_t s) {
    const bool ring = op->profile && op->prof_slots > 1 && op->graphs;
    for (int st = 0; st < nsteps; ++st) {
        if (ring) {
            const int slot = (int)(op->prof_steps % op->prof_slots);
            for (int k = 0; k < 8; ++k)
                NF_CUDA_TRY(cudaGraphExecEventRecordNodeSetEvent(exec, op->graphs->prof_nodes[k],
                                                                 op->prof_ring[8 * slot + k]));
        }
        NF_CUDA_TRY(cudaGraphLaunch(exec, s));
        if (op->profile) ++op->prof_steps;
    }
    return NF_OK;
}

static void destroy_prof_ring(nf_operator *op) {
    for (int i = 0; i < 8 * op->prof_slots; ++i)
        if (op->prof_ring[i]) cudaEventDestroy(op->prof_ring[i]);
    delete[] op->prof_ring;
    op->prof_ring = nullptr;
    op->prof_slots = 0;
}

// Validated forcing for a step: *out is the caller's descriptor, or for NF_FORCE_MMS_SPHERE a
// copy (in *fill) with the Funk-Hecke eigenvalues of the operator's kernel filled in.
static nf_status check_forcing(const nf_operator *op, const nf_forcing *g, const nf_forcing **out,
                               nf_forcing *fill) {
    static const nf_forcing none{NF_FORCE_NONE, nullptr, nullptr, 0, 0, 0, 0, 0, 0, 0, 0};
    if (!g) {
        *out = &none;
        return NF_OK;
    }
    NF_ARG(g->kind == NF_FORCE_NONE || g->kind == NF_FORCE_MMS_EIGEN || g->kind == NF_FORCE_MMS_FLAT ||
               g->kind == NF_FORCE_MMS_SPHERE,
           "unknown forcing kind %d", g->kind);
    if (g->kind == NF_FORCE_MMS_EIGEN) NF_ARG(g->Y1 && g->Y2, "forcing: Y1 and Y2 are required");
    if (g->kind == NF_FORCE_MMS_SPHERE) {
        NF_ARG(op->kp.period == 0.f, "the sphere's manufactured forcing needs the Euclidean (chord) distance");
        NF_ARG(g->c > 0.0 && g->c + std::fabs(g->a0) * 1.5 < 1.0 && g->c - std::fabs(g->a0) * 1.5 > 0.0,
               "sphere manufactured forcing: need 0 < c -+ 1.5 |a0| < 1 (z in (0, 1) on the unit sphere)");
        *fill = *g;
        double lam[3];
        NF_TRY(nf_mms_sphere_eigs(op->kp, lam));
        fill->lam0 = lam[0];
        fill->lam1 = lam[1];
        fill->lam2 = lam[2];
        fill->Y1 = fill->Y2 = nullptr;
        *out = fill;
        return NF_OK;
    }
    if (g->kind == NF_FORCE_MMS_FLAT) {
        NF_ARG(op->kp.period > 0.f, "flat manufactured forcing needs a periodic kernel (period > 0)");
        NF_ARG(g->sigma > 0.0 && g->c > 0.0 && g->c + 1.0 / (2.0 * 3.14159265358979323846 * g->sigma * g->sigma) < 1.0,
               "flat manufactured forcing: need sigma > 0 and 0 < c, c + 1/(2 pi sigma^2) < 1 (z in (0, 1))");
        NF_ARG(std::isfinite(g->radius) && std::isfinite(g->scale), "flat manufactured forcing: radius, scale finite");
    }
    *out = g;
    return NF_OK;
}

}  // namespace nfi

using namespace nfi;

extern "C" {

const char *nf_last_error(void) { return nfi::g_err; }

int nf_version(void) { return (1 << 16) | 0; }

nf_status nf_operator_create(const float *x, const float *q, int64_t n, nf_kernel kp, int path, void *stream,
                             nf_operator **op_out) {
    clear_error();
    NF_ARG(op_out, "op is NULL");
    *op_out = nullptr;
    NF_ARG(x && q, "x and q must be non-NULL device pointers");
    NF_ARG(n >= 1 && n <= (int64_t)1 << 31, "n = %lld out of range", (long long)n);
    NF_ARG(path == NF_MATRIX_FREE || path == NF_DENSE_FP32 || path == NF_DENSE_BF16X2 || path == NF_DENSE_SYM_FP32 ||
               path == NF_DENSE_SYM_BF16X2,
           "unknown path %d", path);
    NF_ARG(std::isfinite(kp.A1) && std::isfinite(kp.A2) && kp.s1 > 0.f && kp.s2 > 0.f && std::isfinite(kp.s1) &&
               std::isfinite(kp.s2),
           "kernel parameters must be finite with s1, s2 > 0");
    NF_ARG(std::isfinite(kp.period) && kp.period >= 0.f, "period must be finite and >= 0");
    cudaStream_t s = as_stream(stream);
    NF_TRY(mf_init_attrs());
    nf_operator *op = new nf_operator();
    op->n = n;
    op->n_pad = round_up(n, kNodePad);
    op->kp = kp;
    op->path = path;
    op->device = device_id();
    auto cleanup = [&](nf_status st) {
        nf_operator_destroy(op);
        return st;
    };
#define CREATE_TRY(expr)                                                                    \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess) return cleanup(cuda_fail(_e, #expr, __FILE__, __LINE__));    \
    } while (0)
    CREATE_TRY(cudaMalloc(&op->x4, op->n_pad * sizeof(float4)));
    CREATE_TRY(cudaMalloc(&op->xyz, 3 * op->n_pad * sizeof(float)));
    CREATE_TRY(cudaMalloc(&op->q, op->n_pad * sizeof(float)));
    CREATE_TRY(cudaMalloc(&op->step_ctr, 64));
    CREATE_TRY(cudaMemsetAsync(op->step_ctr, 0, 64, s));
    op->done_ctr = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(op->step_ctr) + 16);
    op->err = reinterpret_cast<int *>(reinterpret_cast<char *>(op->step_ctr) + 32);
    op->t0_dev = reinterpret_cast<double *>(reinterpret_cast<char *>(op->step_ctr) + 40);
    const float scale = std::sqrt(1.4426950408889634f) / kp.s1;
    pack_nodes_kernel<<<(unsigned)ceil_div(op->n_pad, 256), 256, 0, s>>>(x, q, n, op->n_pad, scale, op->x4, op->xyz,
                                                                         op->q);
    CREATE_TRY(cudaGetLastError());
    if (path == NF_MATRIX_FREE) {
        nf_status st = mf_build_row_order(op, s);
        if (st == NF_OK) st = mf_autotune(op, s);
        if (st != NF_OK) return cleanup(st);
    } else {
        const size_t entries = (size_t)op->n_pad * (size_t)op->n_pad;
        if (path == NF_DENSE_SYM_FP32) {
            CREATE_TRY(cudaMalloc(&op->W32, dense_sym_entries(op->n_pad) * sizeof(float)));
        } else if (path == NF_DENSE_SYM_BF16X2) {  // hi and lo interleaved in one allocation
            CREATE_TRY(cudaMalloc(&op->Whi, 2 * dense_sym_entries(op->n_pad) * sizeof(uint16_t)));
            CREATE_TRY(cudaMalloc(&op->rs, op->n_pad * sizeof(float)));
        } else if (path == NF_DENSE_FP32) {
            CREATE_TRY(cudaMalloc(&op->W32, entries * sizeof(float)));
        } else {
            CREATE_TRY(cudaMalloc(&op->Whi, entries * sizeof(uint16_t)));
            CREATE_TRY(cudaMalloc(&op->Wlo, entries * sizeof(uint16_t)));
            CREATE_TRY(cudaMalloc(&op->rs, op->n_pad * sizeof(float)));
        }
        nf_status st = launch_dense_build(op, s);
        if (st != NF_OK) return cleanup(st);
    }
#undef CREATE_TRY
    *op_out = op;
    return NF_OK;
}

nf_status nf_operator_destroy(nf_operator *op) {
    if (!op) return NF_OK;
    destroy_graphs(op);
    destroy_group(op);
    destroy_prof_ring(op);
    cudaFree(op->x4);
    cudaFree(op->xyz);
    cudaFree(op->rowperm);
    cudaFree(op->cull_pairs);
    cudaFree(op->cull_ptr);
    cudaFree(op->cull_slots);
    cudaFree(op->node_blk);
    cudaFree(op->adj_pairs);
    cudaFree(op->adj_ptr);
    cudaFree(op->adj_slots);
    cudaFree(op->adj_node_blk);
    cudaFree(op->q);
    cudaFree(op->W32);
    cudaFree(op->Whi);
    cudaFree(op->Wlo);
    cudaFree(op->rs);
    cudaFree(op->partial);
    cudaFree(op->g);
    cudaFree(op->U);
    cudaFree(op->ks);
    cudaFree(op->step_ctr);
    delete op;
    return NF_OK;
}

nf_status nf_operator_check(nf_operator *op, void *stream) {
    clear_error();
    NF_ARG(op, "op is NULL");
    NF_CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    int flag = 0;
    NF_CUDA_TRY(cudaMemcpy(&flag, op->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag == DEV_TIMEOUT) return fail(NF_ERR_TIMEOUT, "a bounded device wait timed out");
    if (flag == DEV_NONFINITE) return fail(NF_ERR_NONFINITE, "an RK4 step produced a non-finite state");
    if (flag != 0) return fail(NF_ERR_CUDA, "device error flag %d", flag);
    return NF_OK;
}

nf_status nf_nonlocal_apply(nf_operator *op, const float *u, int B, const float *beta, const float *theta, float *I,
                            void *stream) {
    clear_error();
    NF_ARG(op, "op is NULL");
    NF_ARG(u && beta && theta && I, "u, beta, theta and I must be non-NULL");
    NF_ARG(B >= 1 && B <= 65535, "B = %d out of range", B);
    cudaStream_t s = as_stream(stream);
    if (op->path == NF_GROUPED) {
        NF_ARG(B == group_traj_total(op), "grouped operator: B = %d must equal the group's %d trajectories", B,
               group_traj_total(op));
        NF_TRY(tc_prep(op, u, beta, theta, false, 0, s));
        return tc_launch(op, 0, 0, I, nullptr, beta, theta, 0.0, 0, nullptr, 1, s);
    }
    NF_TRY(ensure_workspace(op, B, nonlocal_splits(op, B)));
    NF_TRY(launch_prep_g(op, u, B, beta, theta, false, s));
    int splits = 1;
    NF_TRY(launch_nonlocal_partial(op, B, s, &splits));
    NF_TRY(launch_reduce_I(op, B, splits, I, s));
    return NF_OK;
}

nf_status nf_rk4_advance(nf_operator *op, float *u, int B, double t0, double dt, int nsteps, const float *beta,
                         const float *theta, const nf_forcing *g, float *ckpt, int C, void *stream) {
    clear_error();
    NF_ARG(op, "op is NULL");
    NF_ARG(u && beta && theta, "u, beta and theta must be non-NULL");
    NF_ARG(B >= 1 && B <= 65535, "B = %d out of range", B);
    NF_ARG(nsteps >= 0, "nsteps must be >= 0");
    NF_ARG(std::isfinite(t0) && std::isfinite(dt), "t0 and dt must be finite");
    NF_ARG(!ckpt || C >= 1, "checkpoint interval C must be >= 1");
    const nf_forcing *F = nullptr;
    nf_forcing Ffill{};
    NF_TRY(check_forcing(op, g, &F, &Ffill));
    cudaStream_t s = as_stream(stream);
    if (op->path == NF_GROUPED) {
        NF_ARG(B == group_traj_total(op), "grouped operator: B = %d must equal the group's %d trajectories", B,
               group_traj_total(op));
        if (F->kind != NF_FORCE_NONE) return fail(NF_ERR_UNSUPPORTED, "grouped operators take no forcing");
        const int64_t tot = group_state_total(op);
        if (ckpt) NF_CUDA_TRY(cudaMemcpyAsync(ckpt, u, sizeof(float) * tot, cudaMemcpyDeviceToDevice, s));
        if (nsteps == 0) return NF_OK;
        cudaGraphExec_t exec = nullptr;
        NF_TRY(rk4_step_graph(op, u, B, dt, beta, theta, *F, ckpt, ckpt ? C : 1, &exec));
        NF_TRY(tc_prep(op, u, beta, theta, true, 0, s));
        NF_TRY(launch_set_clock(op, t0, s));
        return launch_steps(op, exec, nsteps, s);
    }
    if (ckpt) NF_CUDA_TRY(cudaMemcpyAsync(ckpt, u, sizeof(float) * B * op->n, cudaMemcpyDeviceToDevice, s));
    if (nsteps == 0) return NF_OK;
    NF_TRY(ensure_workspace(op, B, nonlocal_splits(op, B)));
    cudaGraphExec_t exec = nullptr;
    NF_TRY(rk4_step_graph(op, u, B, dt, beta, theta, *F, ckpt, ckpt ? C : 1, &exec));
    NF_TRY(launch_prep_g(op, u, B, beta, theta, true, s));
    NF_TRY(launch_set_clock(op, t0, s));
    return launch_steps(op, exec, nsteps, s);
}

nf_status nf_operator_profile(nf_operator *op, int enable) {
    clear_error();
    NF_ARG(op, "op is NULL");
    NF_ARG(enable >= 0 && enable <= 4096, "enable = %d must be 0 (off) or a ring of 1..4096 steps", enable);
    if (enable > 0 && enable != op->prof_slots) {
        destroy_graphs(op);  // captured steps name the old events
        destroy_prof_ring(op);
        op->prof_ring = new cudaEvent_t[8 * (size_t)enable]();
        op->prof_slots = enable;
        for (int i = 0; i < 8 * enable; ++i) NF_CUDA_TRY(cudaEventCreate(&op->prof_ring[i]));
    }
    op->profile = enable != 0;
    op->prof_steps = 0;
    return NF_OK;
}

nf_status nf_operator_kernel_ms_history(nf_operator *op, int steps, float *ms) {
    clear_error();
    NF_ARG(op && ms, "op and ms must be non-NULL");
    NF_ARG(op->profile && op->prof_ring, "profiling is not enabled on this operator");
    NF_ARG(steps >= 1 && steps <= op->prof_slots && steps <= op->prof_steps,
           "steps = %d: %lld profiled steps launched, the ring keeps %d", steps, op->prof_steps, op->prof_slots);
    const long long last = op->prof_steps - 1;
    NF_CUDA_TRY(cudaEventSynchronize(op->prof_ring[8 * (int)(last % op->prof_slots) + 7]));
    for (int k = 0; k < steps; ++k) {
        const cudaEvent_t *ev = op->prof_ring + 8 * (int)((last - steps + 1 + k) % op->prof_slots);
        for (int st = 0; st < 4; ++st) NF_CUDA_TRY(cudaEventElapsedTime(&ms[4 * k + st], ev[2 * st], ev[2 * st + 1]));
    }
    return NF_OK;
}

nf_status nf_operator_kernel_ms(nf_operator *op, float *ms) { return nf_operator_kernel_ms_history(op, 1, ms); }

nf_status nf_selftest_timeout(void *stream) {
    clear_error();
    cudaStream_t s = as_stream(stream);
    int *flag = nullptr;
    NF_CUDA_TRY(cudaMallocAsync(&flag, sizeof(int), s));
    NF_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
    selftest_wait_kernel<<<1, 32, 0, s>>>(flag, 1 << 12);
    NF_CUDA_TRY(cudaGetLastError());
    int h = 0;
    NF_CUDA_TRY(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    NF_CUDA_TRY(cudaFreeAsync(flag, s));
    NF_CUDA_TRY(cudaStreamSynchronize(s));
    if (h == DEV_TIMEOUT) return fail(NF_ERR_TIMEOUT, "bounded wait gave up as expected (self-test)");
    return fail(NF_ERR_CUDA, "self-test wait did not report a timeout (flag %d)", h);
}

nf_status nf_operator_mf_cull(nf_operator *op, int enable, int64_t *live_pairs, int64_t *block_pairs,
                              void *stream) {
    clear_error();
    NF_ARG(op, "op is NULL");
    NF_ARG(op->path == NF_MATRIX_FREE, "culling applies to matrix-free operators");
    return mf_set_cull(op, enable, live_pairs, block_pairs, as_stream(stream));
}

nf_status nf_operator_mf_schedule(nf_operator *op, int schedule) {
    clear_error();
    NF_ARG(op, "op is NULL");
    NF_ARG(op->path == NF_MATRIX_FREE, "the schedule applies to matrix-free operators");
    NF_ARG(schedule >= NF_MF_AUTO && schedule <= NF_MF_SYMMETRIC_1024, "unknown schedule %d", schedule);
    const int blk = schedule == NF_MF_SYMMETRIC_512 ? 512 : (schedule == NF_MF_SYMMETRIC_1024 ? 1024 : op->sym_blk);
    const int sched = schedule >= NF_MF_SYMMETRIC_512 ? NF_MF_SYMMETRIC : schedule;
    destroy_graphs(op);  // captured steps bake in the launch shape
    if (blk != op->sym_blk) op->mf_cull = 0;  // the live-pair lists belong to the old blocks
    op->sym_blk = blk;
    op->mf_sched = sched;
    return NF_OK;
}

nf_status nf_operator_launch_shape(nf_operator *op, int *rows_per_warp, int *tile_cols, int *splits) {
    clear_error();
    NF_ARG(op && rows_per_warp && tile_cols && splits, "arguments must be non-NULL");
    *rows_per_warp = *tile_cols = *splits = -1;
    if (op->path == NF_MATRIX_FREE) mf_launch_shape(op, rows_per_warp, tile_cols, splits);
    return NF_OK;
}

nf_status nf_mms_sphere_eigs(nf_kernel kp, double *lam) {
    clear_error();
    NF_ARG(lam, "lam is NULL");
    NF_ARG(kp.s1 > 0.f && kp.s2 > 0.f, "s1, s2 must be > 0");
    // lam_l = 2 pi int_{-1}^{1} w(sqrt(2 - 2t)) P_l(t) dt; with r^2 = 2(1 - t) each
    // Gaussian gives exp(-a (1 - t)), a = 2 / s^2, and the moments
    //   I_p = int_{-1}^{1} exp(-a (1 - t)) t^p dt  follow by integration by parts.
    lam[0] = lam[1] = lam[2] = 0.0;
    const double amps[2] = {(double)kp.A1, -(double)kp.A2};
    const double sig[2] = {(double)kp.s1, (double)kp.s2};
    for (int h = 0; h < 2; ++h) {
        const double a = 2.0 / (sig[h] * sig[h]);
        const double E = std::exp(-2.0 * a);
        const double I0 = -std::expm1(-2.0 * a) / a;
        const double I1 = (1.0 + E) / a - I0 / a;
        const double I2 = I0 - 2.0 * I1 / a;
        const double twopi = 2.0 * 3.14159265358979323846;
        lam[0] += amps[h] * twopi * I0;
        lam[1] += amps[h] * twopi * I1;
        lam[2] += amps[h] * twopi * 0.5 * (3.0 * I2 - I0);
    }
    return NF_OK;
}

}  // extern "C"
