// nf_internal.cuh -- internal declarations shared by the library's CUDA sources.
// Not part of the C ABI (that is include/nf.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>

#include "../../include/nf.h"

namespace nfi {

// ------------------------------------------------------------------ error plumbing
nf_status fail(nf_status st, const char *fmt, ...);
nf_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);
void clear_error();

#define NF_CUDA_TRY(expr)                                                              \
    do {                                                                               \
        cudaError_t _e = (expr);                                                       \
        if (_e != cudaSuccess) return nfi::cuda_fail(_e, #expr, __FILE__, __LINE__);   \
    } while (0)

#define NF_TRY(expr)                                                                   \
    do {                                                                               \
        nf_status _s = (expr);                                                         \
        if (_s != NF_OK) return _s;                                                    \
    } while (0)

#define NF_ARG(cond, ...)                                                              \
    do {                                                                               \
        if (!(cond)) return nfi::fail(NF_ERR_ARG, __VA_ARGS__);                        \
    } while (0)

// device-side error codes written to an int flag (0 = ok)
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_SINGULAR = 2, DEV_NONFINITE = 3, DEV_BOUNDS = 4 };

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }
inline int64_t ceil_div(int64_t v, int64_t m) { return (v + m - 1) / m; }

int num_sms();
int device_id();

// ------------------------------------------------------------------ PTX helpers
// Bounded waits: a wait that does not complete within the limit reports a timeout
// through the error flag instead of spinning forever.
constexpr long long kSpinLimit = 1ll << 22;  // try_wait polls (~1 s at ~0.25 us per poll)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Returns false if the barrier phase did not complete within kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (long long it = 0; it < kSpinLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Non-suspending poll (test_wait) in a bounded spin, for the single threads that feed the
// tensor core: try_wait may park the thread for a system-dependent interval, which adds
// to every producer / consumer hand-off of a copy pipeline.  ~1 s at ~20 ns per poll.
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_spin_bounded(uint64_t *bar, uint32_t parity) {
    for (long long it = 0; it < (kSpinLimit << 4); ++it)
        if (mbar_test_wait(bar, parity)) return true;
    return false;
}

// 1-D bulk copy global -> shared (TMA unit), completion signalled on `bar`.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// 2^x on the SFU (MUFU.EX2), flush-to-zero: results below 2^-126 become 0.
__device__ __forceinline__ float ex2_sfu(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Doubly periodic distance (§4, Eq. (dist)) on the square of side p: a coordinate
// difference d becomes its nearest image d - p rint(d / p).  rint by adding and removing
// 1.5 * 2^23 (round to nearest even, exact while |d / p| < 2^22), so it stays on the FMA
// pipe.  ip = 1 / p.
constexpr float kRintMagic = 12582912.0f;
__device__ __forceinline__ float wrap1(float d, float p, float ip) {
    const float t = __fsub_rn(__fmaf_rn(d, ip, kRintMagic), kRintMagic);
    return __fmaf_rn(-p, t, d);
}

// Tag selecting the periodic variant of a pair loop at compile time.
template <bool P>
struct PerTag {
    static constexpr bool value = P;
};

// A loop bound known at compile time (full node blocks), interchangeable with a runtime int
// bound (the last, partial block) in templated loops.
template <int V>
struct CInt {
    __device__ constexpr operator int() const { return V; }
};

// Sum of base[k * stride] over k = 0 .. count - 1, added in ascending k.  The loads are
// issued eight at a time before their adds (the order of the adds, hence the result, is that
// of the plain loop), so each thread keeps several slot reads in flight.  base must not be
// written by the calling kernel (read-only cache path).
__device__ __forceinline__ float sum_slots(const float *__restrict__ base, int64_t stride, int count) {
    float s = 0.f;
    int k = 0;
    for (; k + 8 <= count; k += 8) {
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = __ldg(base + (int64_t)(k + j) * stride);
#pragma unroll
        for (int j = 0; j < 8; ++j) s += v[j];
    }
    for (; k < count; ++k) s += __ldg(base + (int64_t)k * stride);
    return s;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void set_dev_error(int *flag, int code) {
    if (flag) atomicCAS(flag, 0, code);
}

__device__ __forceinline__ float bf16_bits_to_float(uint32_t h) { return __uint_as_float(h << 16); }

}  // namespace nfi

// ---------------------------------------------------------------------- operator
// Node data are padded to n_pad (a multiple of kNodePad) with q = 0, so padded
// columns contribute nothing and every tile is full.
constexpr int64_t kNodePad = 1024;

struct nf_graph_cache;
struct nf_group_state;

// internal path id of a grouped operator (several bf16 hi+lo operators, tensor-core GEMM)
constexpr int NF_GROUPED = 3;

struct nf_operator {
    int64_t n = 0, n_pad = 0;
    nf_kernel kp{};
    int path = 0;
    int device = 0;
    float4 *x4 = nullptr;    // n_pad: (x, y, z, 0)
    float *xyz = nullptr;    // 3 x n_pad: coordinates times sqrt(log2 e)/s1, structure of arrays
    int mf_variant = -1;     // launch shape of the packed pair kernel
    int mf_sym_r = 8;        // rows per warp of the symmetric single-trajectory kernel (autotuned)
    int adj_r = 0;           // rows per warp of the adjoint pair kernel (0: not yet timed; 4 or 8)
    int adj_blk = 0;         // its node block (0: not yet timed; 1024 or 512)
    int mf_sched = 0;        // NF_MF_AUTO / NF_MF_SYMMETRIC / NF_MF_PACKED
    int sym_blk = 1024;      // node block of the symmetric kernel (1024, or 512 when autotuned faster)
    int planar = 0;          // every node has the same z: the symmetric kernel drops the z terms
    // block-pair culling of the symmetric kernel (opt-in, nf_operator_mf_cull)
    int mf_cull = 0;
    int *cull_pairs = nullptr;   // live block-pair indices (ascending)
    int64_t cull_live = 0;
    int *cull_ptr = nullptr;     // nb + 1: each node block's live slots in cull_slots
    int *cull_slots = nullptr;   // ascending per block
    int *node_blk = nullptr;     // n_pad: Morton block of each node
    int *adj_pairs = nullptr;    // the adjoint kernel's live pairs of 1,024-node blocks (both Gaussians)
    int64_t adj_live = 0;
    int *adj_ptr = nullptr, *adj_slots = nullptr, *adj_node_blk = nullptr;
    int *rowperm = nullptr;  // n_pad: row order of the packed pair kernel (Morton order of the nodes)
    float *q = nullptr;      // n_pad, zero padded
    // dense planes (row-major, leading dimension ld = n_pad)
    float *W32 = nullptr;        // W diag(q), FP32
    uint16_t *Whi = nullptr;     // bf16 bits of (W diag(q))_ij / s_i, high part (blocked layout)
    uint16_t *Wlo = nullptr;     // bf16 bits of the residual (blocked layout)
    float *rs = nullptr;         // s_i, powers of two (symmetric bf16 planes: K_ij = s_i s_j (hi + lo))
    // workspace owned by the handle
    float *partial = nullptr;    // [split][B][n_pad]
    size_t partial_cap = 0;
    float *g = nullptr;          // [B][n_pad]: q_j f(U_j) (matrix-free) or f(U_j) (dense)
    float *U = nullptr;          // [B][n]: current stage input
    float *ks = nullptr;         // [B][n]: RK4 slope accumulator
    size_t state_cap = 0;        // elements of U / ks
    size_t g_cap = 0;
    long long *step_ctr = nullptr;  // device step counter for graph replay
    unsigned *done_ctr = nullptr;   // last-block-done counter
    int *err = nullptr;             // device error flag
    double *t0_dev = nullptr;       // start time of the current nf_rk4_advance call
    nf_graph_cache *graphs = nullptr;
    nf_group_state *group = nullptr;   // grouped operators only (members are not owned)
    // live kernel timing: events recorded around each stage's nonlocal launches.  The step
    // graph is captured with slot 0's eight events; before each replay the graph's event
    // nodes are pointed at slot (step % prof_slots), so the last prof_slots steps keep
    // their own timings until they are read.
    bool profile = false;
    cudaEvent_t *prof_ring = nullptr;  // prof_slots x 8
    int prof_slots = 0;
    long long prof_steps = 0;          // profiled steps launched since profiling was enabled
};

namespace nfi {

// Blocked layout of the bf16 planes: 128-row x 64-column blocks of 16 KB, each stored row by
// row (128 bytes per row), blocks ordered by row block, then column block.  A tensor-core
// operand tile (128 rows x 64 K) is one contiguous 16 KB read; a row's 64-column pieces lie
// 16 KB apart.  n_pad is a multiple of 1024, so the blocks tile the padded matrix exactly.
constexpr int kBlkRows = 128, kBlkCols = 64;
__host__ __device__ __forceinline__ int64_t blocked_offset(int64_t i, int64_t j, int64_t n_pad) {
    return (((i >> 7) * (n_pad >> 6) + (j >> 6)) << 13) + ((i & 127) << 6) + (j & 63);
}

// ---------------------------------------------------------------- launch plans
struct SplitPlan {
    int rows_per_block;   // rows of I per block
    int64_t row_blocks;
    int splits;           // j-range splits (blockIdx.y)
    int64_t jchunk;       // columns per split, a multiple of the tile width
};
SplitPlan plan_splits(int64_t n_pad, int rows_per_block, int tile_cols, int resident_blocks_per_sm,
                      int max_splits = 64);

nf_status ensure_workspace(nf_operator *op, int B, int splits);

// matrix-free / dense nonlocal launches (g must hold q f(U) / f(U) for B trajectories)
nf_status mf_init_attrs();
nf_status mf_build_row_order(nf_operator *op, cudaStream_t s);
SplitPlan mf_plan(nf_operator *op);     // column splits of the multi-trajectory matrix-free launches
int mf_splits(nf_operator *op, int B);  // partial-sum slots of a matrix-free launch over B trajectories
int64_t sym_pair_count(const nf_operator *op);  // block pairs of the symmetric kernels
int sym_slots(const nf_operator *op);   // node blocks of the symmetric schedule (W nu slots)
int adj_slots(const nf_operator *op);   // node blocks of the adjoint kernel (its W nu slots)
int64_t adj_pair_capacity(const nf_operator *op);  // block pairs / slots of the adjoint kernel's
int adj_slot_capacity(const nf_operator *op);      // smallest block (512): scratch sizes
nf_status mf_set_cull(nf_operator *op, int enable, int64_t *live, int64_t *total, cudaStream_t s);
nf_status launch_adj_cull_reduce(nf_operator *op, float *wpart, int B, int b, cudaStream_t s);
nf_status launch_adj_sym(nf_operator *op, const float2 *vg, int B, int b, float *wpart, float *gpart,
                         float *r2_phys, cudaStream_t s);
nf_status adj_autotune(nf_operator *op, const float2 *vg, int B, float *wpart, float *gpart, cudaStream_t s);
nf_status mf_autotune(nf_operator *op, cudaStream_t s);
void mf_launch_shape(nf_operator *op, int *R, int *TJ, int *splits);
nf_status launch_mf_pair(nf_operator *op, int B, cudaStream_t s, int *splits_out);
SplitPlan plan_mf_pair_single(int64_t n_pad, int max_splits);
nf_status launch_mf_pair_single(const float4 *x4, const float *g, int64_t n_pad, const nf_kernel &k, int max_splits,
                                float *partial, int *err, cudaStream_t s, int *splits_out);
nf_status launch_dense_gemv(nf_operator *op, int B, cudaStream_t s, int *splits_out);
int dense_splits(nf_operator *op, int B);    // partial-sum slots of a dense launch over B trajectories
nf_status dense_init_attrs();
size_t dense_sym_entries(int64_t n_pad);     // stored entries of the symmetric blocked matrix
// q is applied on the vector side (g = q o f) unless it is folded into a dense operator
inline bool q_on_vector(const nf_operator *op) {
    return op->path == NF_MATRIX_FREE || op->path == NF_DENSE_SYM_FP32 || op->path == NF_DENSE_SYM_BF16X2;
}
nf_status launch_dense_build(nf_operator *op, cudaStream_t s);

// elementwise kernels
nf_status launch_prep_g(nf_operator *op, const float *u, int B, const float *beta, const float *theta,
                        bool copy_to_U, cudaStream_t s);
nf_status launch_reduce_I(nf_operator *op, int B, int splits, float *I, cudaStream_t s);

struct StageParams {
    float *u;              // B x n in/out
    const float *beta, *theta;
    nf_forcing forcing;
    double dt;             // t0 is read from the operator's device clock
    int stage;             // 1..4
    float *ckpt;
    int C;
    int splits;
};
nf_status launch_stage(nf_operator *op, int B, const StageParams &p, cudaStream_t s);
nf_status launch_set_clock(nf_operator *op, double t0, cudaStream_t s);

// nonlocal sum of the current g into partial (path dispatch)
nf_status launch_nonlocal_partial(nf_operator *op, int B, cudaStream_t s, int *splits_out);
int nonlocal_splits(nf_operator *op, int B);  // partial-sum slots of launch_nonlocal_partial

void destroy_graphs(nf_operator *op);

// grouped tensor-core path (nf_tc.cu)
void destroy_group(nf_operator *op);
int group_traj_total(const nf_operator *op);
int64_t group_state_total(const nf_operator *op);
nf_status tc_prep(nf_operator *op, const float *u, const float *beta, const float *theta, bool copy_U, int buffer,
                  cudaStream_t s);
nf_status tc_launch(nf_operator *op, int parity, int mode, float *I, float *u, const float *beta, const float *theta,
                    double dt, int stage, float *ckpt, int C, cudaStream_t s);

}  // namespace nfi
