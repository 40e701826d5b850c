// nf_mf.cu -- matrix-free nonlocal sum (§2.2, Eq. (2.9)) and the fused RK4 stage
// kernel.
//
// Pair kernel.  I[b, i] = sum_j w(|x_i - x_j|) g[b, j], g = q o f(U) (FP32), with the
// Mexican-hat kernel w(r) = A1 exp(-r^2/s1^2) - A2 exp(-r^2/s2^2).  Work is split
// into items (row block, column split): each warp owns R rows (coordinates in
// registers); its lanes stride over the columns of the split; column tiles of
// MF_TJ nodes (x, y, z and the NB trajectories' g values) are staged into shared
// memory by the TMA bulk-copy unit, double buffered on mbarriers.  Per pair:
// 3 FADD + FMUL + 2 FFMA (r^2), 2 FMUL (exponent scaling), 2 MUFU.EX2, and 2 FFMA
// (NB = 1: separate e1 and e2 accumulators) or FMUL + FFMA + NB FFMA (NB > 1).
// Each warp reduces its rows with shuffles and writes one partial sum per
// (split, trajectory, row); the stage kernel (or the reduce kernel) adds the
// splits in a fixed order, so results are deterministic.
#include "nf_internal.cuh"

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>

namespace nfi {

constexpr int MF_THREADS = 256;
constexpr int MF_WARPS = MF_THREADS / 32;
constexpr int MF_TJ = 512;  // columns per shared-memory tile; divides kNodePad
static_assert(kNodePad % MF_TJ == 0, "tile must divide the node padding");

template <int NB>
struct MfSmem {
    float4 xs[2][MF_TJ];
    float gs[2][NB][MF_TJ];
    uint64_t bar[2];
};

template <int NB, int R>
__global__ void __launch_bounds__(MF_THREADS)
mf_pair_kernel(const float4 *__restrict__ x4, const float *__restrict__ g, int64_t n_pad, int B, int b_base,
               int64_t jchunk, float c1, float c2, float A1, float A2, float *__restrict__ partial,
               int *__restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MfSmem<NB> &sm = *reinterpret_cast<MfSmem<NB> *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int split = blockIdx.y;
    const int b0 = b_base + blockIdx.z * NB;
    const int64_t j0 = (int64_t)split * jchunk;
    const int64_t j1 = min(n_pad, j0 + jchunk);
    const int ntiles = (int)((j1 - j0) / MF_TJ);
    const int64_t row0 = ((int64_t)blockIdx.x * MF_WARPS + warp) * R;
    constexpr uint32_t kTileBytes = MF_TJ * 16 + NB * MF_TJ * 4;

    if (tid == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();

    auto issue = [&](int t) {
        const int buf = t & 1;
        const int64_t jt = j0 + (int64_t)t * MF_TJ;
        mbar_arrive_expect_tx(&sm.bar[buf], kTileBytes);
        bulk_g2s(sm.xs[buf], x4 + jt, MF_TJ * 16, &sm.bar[buf]);
#pragma unroll
        for (int b = 0; b < NB; ++b) bulk_g2s(sm.gs[buf][b], g + (int64_t)(b0 + b) * n_pad + jt, MF_TJ * 4, &sm.bar[buf]);
    };
    if (tid == 0) {
        if (ntiles > 0) issue(0);
        if (ntiles > 1) issue(1);
    }

    float xi[R], yi[R], zi[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float4 p = x4[row0 + r];
        xi[r] = p.x;
        yi[r] = p.y;
        zi[r] = p.z;
    }
    constexpr int NA = (NB == 1) ? 2 : NB;  // NB == 1: separate e1 / e2 accumulators
    float acc[R][NA];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int a = 0; a < NA; ++a) acc[r][a] = 0.f;

    bool timed_out = false;
    for (int t = 0; t < ntiles; ++t) {
        const int buf = t & 1;
        const bool ok = mbar_wait_bounded(&sm.bar[buf], (uint32_t)((t >> 1) & 1));
        // Uniform decision; this barrier also certifies that every warp has finished
        // tile t-1, whose buffer the next issue overwrites.
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        if (tid == 0 && t >= 1 && t + 1 < ntiles) issue(t + 1);
        const float4 *xs = sm.xs[buf];
#pragma unroll 4
        for (int jj = lane; jj < MF_TJ; jj += 32) {
            const float4 xj = xs[jj];
            float gb[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) gb[b] = sm.gs[buf][b][jj];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float dx = xi[r] - xj.x, dy = yi[r] - xj.y, dz = zi[r] - xj.z;
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                const float e1 = ex2_sfu(r2 * c1);
                const float e2 = ex2_sfu(r2 * c2);
                if constexpr (NB == 1) {
                    acc[r][0] = fmaf(e1, gb[0], acc[r][0]);
                    acc[r][1] = fmaf(e2, gb[0], acc[r][1]);
                } else {
                    const float w = fmaf(A1, e1, -A2 * e2);
#pragma unroll
                    for (int b = 0; b < NB; ++b) acc[r][b] = fmaf(w, gb[b], acc[r][b]);
                }
            }
        }
    }
    if (timed_out) {
        if (tid == 0) set_dev_error(err, DEV_TIMEOUT);
        // let any copy still in flight land before the block's shared memory is released
        if (tid == 0)
            for (int b = 0; b < 2; ++b) (void)mbar_wait_bounded(&sm.bar[b], 0), (void)mbar_wait_bounded(&sm.bar[b], 1);
        return;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            float v = (NB == 1) ? (A1 * acc[r][0] - A2 * acc[r][1]) : acc[r][b];
            v = warp_sum(v);
            if (lane == 0) partial[((int64_t)split * B + (b0 + b)) * n_pad + row0 + r] = v;
        }
    }
}

// ----------------------------------------------------------------------------
// Single-trajectory variant on packed FP32 pairs (f32x2: one instruction, two lanes of
// the FMA pipe).  Column tiles are staged as structure-of-arrays (x, y, z, g), so a
// lane reads two adjacent columns with one 8-byte load; each row's coordinates are held
// duplicated in a 64-bit register pair.  Per two pairs: 3 SUB2, MUL2 + 2 FMA2 (r^2),
// 2 MUL2 (exponent scaling), 4 MUFU.EX2, 2 FMA2 -- 7 issue slots per pair instead of 12,
// the same FMA-pipe lane count, the same rounding as the scalar kernel.
typedef unsigned long long u64;
__device__ __forceinline__ u64 f2_sub(u64 a, u64 b) {
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 f2_mul(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 f2_fma(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 f2_pack(float lo, float hi) {
    u64 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ void f2_unpack(u64 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 f2_ex2(u64 a) {
    float lo, hi;
    f2_unpack(a, lo, hi);
    return f2_pack(ex2_sfu(lo), ex2_sfu(hi));
}

template <int TJ>
struct MfPackedSmem {
    float xs[2][TJ], ys[2][TJ], zs[2][TJ], gs[2][TJ];
    uint64_t bar[2];
};

// xyz: pre-scaled coordinates as structure of arrays [x(n_pad) | y(n_pad) | z(n_pad)],
// multiplied by sqrt(log2 e) / s1; g_all: B x n_pad firing rates (times q).
template <int R, int TJ>
__global__ void __launch_bounds__(MF_THREADS)
mf_pair_packed_kernel(const float *__restrict__ xyz, const float *__restrict__ g_all, int64_t n_pad, int B,
                      int b_base, int64_t jchunk, float k2, float A1, float A2, float *__restrict__ partial,
                      int *__restrict__ err) {
    __shared__ __align__(128) MfPackedSmem<TJ> sm;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int split = blockIdx.y;
    const int64_t j0 = (int64_t)split * jchunk;
    const int64_t j1 = min(n_pad, j0 + jchunk);
    const int ntiles = (int)((j1 - j0) / TJ);
    const int64_t row0 = ((int64_t)blockIdx.x * MF_WARPS + warp) * R;
    constexpr uint32_t kTileBytes = 4 * TJ * 4;
    const float *X = xyz, *Y = xyz + n_pad, *Z = xyz + 2 * n_pad;
    const int b = b_base + blockIdx.z;
    const float *g = g_all + (int64_t)b * n_pad;
    if (tid == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](int t) {
        const int buf = t & 1;
        const int64_t jt = j0 + (int64_t)t * TJ;
        mbar_arrive_expect_tx(&sm.bar[buf], kTileBytes);
        bulk_g2s(sm.xs[buf], X + jt, TJ * 4, &sm.bar[buf]);
        bulk_g2s(sm.ys[buf], Y + jt, TJ * 4, &sm.bar[buf]);
        bulk_g2s(sm.zs[buf], Z + jt, TJ * 4, &sm.bar[buf]);
        bulk_g2s(sm.gs[buf], g + jt, TJ * 4, &sm.bar[buf]);
    };
    if (tid == 0) {
        if (ntiles > 0) issue(0);
        if (ntiles > 1) issue(1);
    }
    u64 xi[R], yi[R], zi[R], a1[R], a2[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float x = X[row0 + r], y = Y[row0 + r], z = Z[row0 + r];
        xi[r] = f2_pack(x, x);
        yi[r] = f2_pack(y, y);
        zi[r] = f2_pack(z, z);
        a1[r] = 0ull;
        a2[r] = 0ull;
    }
    // coordinates arrive pre-scaled by sqrt(log2(e)) / s1, so r2s = r^2 log2(e) / s1^2:
    // e1 = 2^(-r2s), e2 = 2^(-k2 r2s) with k2 = s1^2 / s2^2
    const u64 nk2 = f2_pack(-k2, -k2);
    bool timed_out = false;
    for (int t = 0; t < ntiles; ++t) {
        const int buf = t & 1;
        const bool ok = mbar_wait_bounded(&sm.bar[buf], (uint32_t)((t >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        if (tid == 0 && t >= 1 && t + 1 < ntiles) issue(t + 1);
        const u64 *xs = reinterpret_cast<const u64 *>(sm.xs[buf]);
        const u64 *ys = reinterpret_cast<const u64 *>(sm.ys[buf]);
        const u64 *zs = reinterpret_cast<const u64 *>(sm.zs[buf]);
        const u64 *gs = reinterpret_cast<const u64 *>(sm.gs[buf]);
#pragma unroll 2
        for (int jp = lane; jp < TJ / 2; jp += 32) {
            const u64 xj = xs[jp], yj = ys[jp], zj = zs[jp], gj = gs[jp];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const u64 dx = f2_sub(xi[r], xj), dy = f2_sub(yi[r], yj), dz = f2_sub(zi[r], zj);
                const u64 r2s = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
                float s0, s1v;
                f2_unpack(r2s, s0, s1v);
                const u64 e1 = f2_pack(ex2_sfu(-s0), ex2_sfu(-s1v));
                const u64 e2 = f2_ex2(f2_mul(r2s, nk2));
                a1[r] = f2_fma(e1, gj, a1[r]);
                a2[r] = f2_fma(e2, gj, a2[r]);
            }
        }
    }
    if (timed_out) {
        if (tid == 0) {
            set_dev_error(err, DEV_TIMEOUT);
            for (int b = 0; b < 2; ++b) (void)mbar_wait_bounded(&sm.bar[b], 0), (void)mbar_wait_bounded(&sm.bar[b], 1);
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float p0, p1, q0, q1;
        f2_unpack(a1[r], p0, p1);
        f2_unpack(a2[r], q0, q1);
        float v = A1 * (p0 + p1) - A2 * (q0 + q1);
        v = warp_sum(v);
        if (lane == 0) partial[((int64_t)split * B + b) * n_pad + row0 + r] = v;
    }
}

// ----------------------------------------------------------------------------
// split planner: (row blocks x column splits) items of equal cost; pick the number
// of splits that best fills whole waves of resident blocks.
SplitPlan plan_splits(int64_t n_pad, int rows_per_block, int tile_cols, int resident_blocks_per_sm) {
    SplitPlan p{};
    p.rows_per_block = rows_per_block;
    p.row_blocks = n_pad / rows_per_block;
    const int64_t tiles = n_pad / tile_cols;
    const int64_t slots = (int64_t)num_sms() * std::max(1, resident_blocks_per_sm);
    double best = -1.0;
    int best_s = 1;
    const int64_t smax = std::min<int64_t>(tiles, 64);
    for (int64_t s = 1; s <= smax; ++s) {
        const int64_t per = ceil_div(tiles, s);
        const int64_t s_eff = ceil_div(tiles, per);
        if (s_eff != s) continue;
        const int64_t items = p.row_blocks * s_eff;
        const int64_t waves = ceil_div(items, slots);
        double eff = (double)items / (double)(waves * slots);
        // each extra split costs a little (prologue, partial traffic): prefer fewer
        eff -= 0.002 * (double)s;
        if (eff > best + 1e-9) {
            best = eff;
            best_s = (int)s;
        }
        if (items >= 16 * slots) break;  // enough waves that the tail is negligible
    }
    p.splits = best_s;
    p.jchunk = ceil_div(tiles, best_s) * tile_cols;
    return p;
}

template <int NB, int R>
static cudaError_t set_mf_attr() {
    return cudaFuncSetAttribute(mf_pair_kernel<NB, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(MfSmem<NB>));
}

// Opt every pair-kernel instance into its shared-memory size (outside any capture).
nf_status mf_init_attrs() {
    NF_CUDA_TRY((set_mf_attr<1, 2>()));
    NF_CUDA_TRY((set_mf_attr<2, 2>()));
    NF_CUDA_TRY((set_mf_attr<4, 2>()));
    NF_CUDA_TRY((set_mf_attr<8, 2>()));
    NF_CUDA_TRY((set_mf_attr<1, 4>()));
    NF_CUDA_TRY((set_mf_attr<2, 4>()));
    NF_CUDA_TRY((set_mf_attr<4, 4>()));
    NF_CUDA_TRY((set_mf_attr<8, 4>()));
    return NF_OK;
}

template <int NB, int R>
static nf_status launch_mf_group(nf_operator *op, int B, int b_base, int groups, const SplitPlan &pl,
                                 cudaStream_t s) {
    const size_t smem = sizeof(MfSmem<NB>);
    const float L2E = 1.4426950408889634f;
    const nf_kernel &k = op->kp;
    const float c1 = -L2E / (k.s1 * k.s1), c2 = -L2E / (k.s2 * k.s2);
    dim3 grid((unsigned)pl.row_blocks, (unsigned)pl.splits, (unsigned)groups);
    mf_pair_kernel<NB, R><<<grid, MF_THREADS, smem, s>>>(op->x4, op->g, op->n_pad, B, b_base, pl.jchunk, c1, c2,
                                                         k.A1, k.A2, op->partial, op->err);
    NF_CUDA_TRY(cudaGetLastError());
    return NF_OK;
}

template <int NB, int R>
static int mf_resident() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, mf_pair_kernel<NB, R>, MF_THREADS, sizeof(MfSmem<NB>));
    return std::max(nb, 1);
}

// Launch shapes of the packed kernel the autotuner chooses from: rows per warp, tile width.
struct MfVariant {
    int R, TJ;
};
constexpr MfVariant kMfVariants[] = {{2, 512}, {4, 512}, {4, 1024}, {8, 1024}};
constexpr int kNumMfVariants = 4;

template <int R, int TJ>
static int packed_resident() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, mf_pair_packed_kernel<R, TJ>, MF_THREADS, 0);
    return std::max(nb, 1);
}

static int variant_resident(int v) {
    switch (v) {
        case 0: return packed_resident<2, 512>();
        case 1: return packed_resident<4, 512>();
        case 2: return packed_resident<4, 1024>();
        default: return packed_resident<8, 1024>();
    }
}

template <int R, int TJ>
static void launch_packed(nf_operator *op, int B, int b_base, int groups, const SplitPlan &pl, cudaStream_t s) {
    const nf_kernel &k = op->kp;
    const float k2 = (k.s1 * k.s1) / (k.s2 * k.s2);
    dim3 grid((unsigned)pl.row_blocks, (unsigned)pl.splits, (unsigned)groups);
    mf_pair_packed_kernel<R, TJ><<<grid, MF_THREADS, 0, s>>>(op->xyz, op->g, op->n_pad, B, b_base, pl.jchunk, k2, k.A1,
                                                             k.A2, op->partial, op->err);
}

static nf_status launch_mf_packed(nf_operator *op, int B, int b_base, int groups, const SplitPlan &pl,
                                  cudaStream_t s) {
    switch (op->mf_variant) {
        case 0: launch_packed<2, 512>(op, B, b_base, groups, pl, s); break;
        case 1: launch_packed<4, 512>(op, B, b_base, groups, pl, s); break;
        case 2: launch_packed<4, 1024>(op, B, b_base, groups, pl, s); break;
        default: launch_packed<8, 1024>(op, B, b_base, groups, pl, s); break;
    }
    NF_CUDA_TRY(cudaGetLastError());
    return NF_OK;
}

// Default before (or without) autotuning: small node sets want more, smaller blocks.
static int default_variant(int64_t n_pad) { return n_pad >= 16384 ? 1 : 0; }

static SplitPlan variant_plan(int64_t n_pad, int v) {
    return plan_splits(n_pad, MF_WARPS * kMfVariants[v].R, kMfVariants[v].TJ, variant_resident(v));
}

SplitPlan mf_plan(nf_operator *op) {
    if (op->mf_variant < 0) op->mf_variant = default_variant(op->n_pad);
    return variant_plan(op->n_pad, op->mf_variant);
}

void mf_launch_shape(nf_operator *op, int *R, int *TJ, int *splits) {
    const SplitPlan pl = mf_plan(op);
    *R = kMfVariants[op->mf_variant].R;
    *TJ = kMfVariants[op->mf_variant].TJ;
    *splits = pl.splits;
}

// Rows per warp of the scalar multi-trajectory kernel (2 or 4 are instantiated).
static int mf_rows_per_warp(int64_t n_pad) { return n_pad >= 16384 ? 4 : 2; }

// Time every launch shape once on this operator's size and keep the fastest (cached
// per padded size and device).  Runs outside any stream capture.
nf_status mf_autotune(nf_operator *op, cudaStream_t s) {
    static std::mutex mu;
    static std::map<std::pair<int, int64_t>, int> cache;
    const auto key = std::make_pair(op->device, op->n_pad);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            op->mf_variant = it->second;
            return NF_OK;
        }
    }
    int max_splits = 1;
    for (int v = 0; v < kNumMfVariants; ++v) max_splits = std::max(max_splits, variant_plan(op->n_pad, v).splits);
    NF_TRY(ensure_workspace(op, 1, max_splits));
    cudaEvent_t e0, e1;
    NF_CUDA_TRY(cudaEventCreate(&e0));
    NF_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_v = default_variant(op->n_pad);
    for (int v = 0; v < kNumMfVariants; ++v) {
        op->mf_variant = v;
        const SplitPlan pl = variant_plan(op->n_pad, v);
        NF_TRY(launch_mf_packed(op, 1, 0, 1, pl, s));  // warm-up
        NF_CUDA_TRY(cudaEventRecord(e0, s));
        for (int rep = 0; rep < 2; ++rep) NF_TRY(launch_mf_packed(op, 1, 0, 1, pl, s));
        NF_CUDA_TRY(cudaEventRecord(e1, s));
        NF_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        NF_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
            best = ms;
            best_v = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    op->mf_variant = best_v;
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = best_v;
    return NF_OK;
}

nf_status launch_mf_pair(nf_operator *op, int B, cudaStream_t s, int *splits_out) {
    // the column splits (and so the partial-sum layout) come from the packed kernel's
    // plan; the scalar multi-trajectory kernels block rows their own way over the same splits
    const SplitPlan pl = mf_plan(op);
    const int R = mf_rows_per_warp(op->n_pad);
    SplitPlan spl = pl;
    spl.rows_per_block = MF_WARPS * R;
    spl.row_blocks = op->n_pad / spl.rows_per_block;
    int b = 0;
    auto run = [&](int nb) -> nf_status {
        const int groups = (B - b) / nb;
        if (groups <= 0) return NF_OK;
        nf_status st = NF_OK;
        if (nb == 1) {
            st = launch_mf_packed(op, B, b, groups, pl, s);
        } else if (R == 4) {
            switch (nb) {
                case 8: st = launch_mf_group<8, 4>(op, B, b, groups, spl, s); break;
                case 4: st = launch_mf_group<4, 4>(op, B, b, groups, spl, s); break;
                default: st = launch_mf_group<2, 4>(op, B, b, groups, spl, s); break;
            }
        } else {
            switch (nb) {
                case 8: st = launch_mf_group<8, 2>(op, B, b, groups, spl, s); break;
                case 4: st = launch_mf_group<4, 2>(op, B, b, groups, spl, s); break;
                default: st = launch_mf_group<2, 2>(op, B, b, groups, spl, s); break;
            }
        }
        b += groups * nb;
        return st;
    };
    NF_TRY(run(8));
    NF_TRY(run(4));
    NF_TRY(run(2));
    NF_TRY(run(1));
    *splits_out = pl.splits;
    return NF_OK;
}

// Single-trajectory pair sums into caller-provided buffers (x4, g padded to n_pad,
// partial [splits][n_pad]); the split count is capped at max_splits.
nf_status launch_mf_pair_single(const float4 *x4, const float *g, int64_t n_pad, const nf_kernel &k, int max_splits,
                                float *partial, int *err, cudaStream_t s, int *splits_out) {
    const int R = mf_rows_per_warp(n_pad);
    SplitPlan pl = plan_splits(n_pad, MF_WARPS * R, MF_TJ, R == 4 ? mf_resident<1, 4>() : mf_resident<1, 2>());
    if (pl.splits > max_splits) {
        const int64_t tiles = n_pad / MF_TJ;
        const int64_t per = ceil_div(tiles, max_splits);
        pl.jchunk = per * MF_TJ;
        pl.splits = (int)ceil_div(tiles, per);
    }
    const float L2E = 1.4426950408889634f;
    const float c1 = -L2E / (k.s1 * k.s1), c2 = -L2E / (k.s2 * k.s2);
    dim3 grid((unsigned)pl.row_blocks, (unsigned)pl.splits, 1);
    if (R == 4)
        mf_pair_kernel<1, 4><<<grid, MF_THREADS, sizeof(MfSmem<1>), s>>>(x4, g, n_pad, 1, 0, pl.jchunk, c1, c2, k.A1,
                                                                      k.A2, partial, err);
    else
        mf_pair_kernel<1, 2><<<grid, MF_THREADS, sizeof(MfSmem<1>), s>>>(x4, g, n_pad, 1, 0, pl.jchunk, c1, c2, k.A1,
                                                                      k.A2, partial, err);
    NF_CUDA_TRY(cudaGetLastError());
    *splits_out = pl.splits;
    return NF_OK;
}

// ----------------------------------------------------------------------------
// Elementwise kernels.

__device__ __forceinline__ float firing_rate(float u, float beta, float theta) {
    return 1.0f / (1.0f + expf(-beta * (u - theta)));
}

// g[b, j] = q_j f_b(u[b, j]) (q == nullptr: f alone);  optionally U = u.
__global__ void prep_g_kernel(const float *__restrict__ u, int64_t n, int64_t n_pad, int B,
                              const float *__restrict__ q, const float *__restrict__ beta,
                              const float *__restrict__ theta, float *__restrict__ g, float *__restrict__ U) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)B * n) return;
    const int b = (int)(idx / n);
    const int64_t j = idx - (int64_t)b * n;
    const float uv = u[idx];
    const float f = firing_rate(uv, beta[b], theta[b]);
    g[(int64_t)b * n_pad + j] = q ? q[j] * f : f;
    if (U) U[idx] = uv;
}

nf_status launch_prep_g(nf_operator *op, const float *u, int B, const float *beta, const float *theta,
                        bool copy_to_U, cudaStream_t s) {
    const int64_t tot = (int64_t)B * op->n;
    const int T = 256;
    const bool mf = (op->path == NF_MATRIX_FREE);
    prep_g_kernel<<<(unsigned)ceil_div(tot, T), T, 0, s>>>(u, op->n, op->n_pad, B, mf ? op->q : nullptr, beta,
                                                          theta, op->g, copy_to_U ? op->U : nullptr);
    NF_CUDA_TRY(cudaGetLastError());
    return NF_OK;
}

__global__ void reduce_I_kernel(const float *__restrict__ partial, int splits, int64_t n, int64_t n_pad, int B,
                                const float *__restrict__ rs, float *__restrict__ I) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)B * n) return;
    const int b = (int)(idx / n);
    const int64_t i = idx - (int64_t)b * n;
    float acc = 0.f;
    for (int sp = 0; sp < splits; ++sp) acc += partial[((int64_t)sp * B + b) * n_pad + i];
    I[idx] = rs ? acc * rs[i] : acc;
}

nf_status launch_reduce_I(nf_operator *op, int B, int splits, float *I, cudaStream_t s) {
    const int64_t tot = (int64_t)B * op->n;
    const int T = 256;
    const float *rs = (op->path == NF_DENSE_BF16X2) ? op->rs : nullptr;
    reduce_I_kernel<<<(unsigned)ceil_div(tot, T), T, 0, s>>>(op->partial, splits, op->n, op->n_pad, B, rs, I);
    NF_CUDA_TRY(cudaGetLastError());
    return NF_OK;
}

// ----------------------------------------------------------------------------
// Fused RK4 stage: I = sum of splits; k_s = -U_s + I + gamma(t_s); RK4 bookkeeping;
// next stage input and its g.  On the last stage the last block advances the
// device step counter, so one captured step can be replayed.
struct StageKArgs {
    const float *partial;
    int splits;
    int64_t n, n_pad;
    int B;
    float *u, *U, *ks, *g;
    const float *q;     // matrix-free: g = q f; dense: g = f (q lives in W)
    const float *rs;    // BF16X2 row scale, or null
    const float *beta, *theta;
    nf_forcing F;
    const double *t0;
    double dt;
    int stage;
    long long *step_ctr;
    unsigned *done_ctr;
    float *ckpt;
    int C;
};

__device__ __forceinline__ double forcing_value(const nf_forcing &F, int64_t i, double t, float beta,
                                                float theta) {
    if (F.kind != NF_FORCE_MMS_EIGEN) return 0.0;
    const double Y1 = F.Y1[i], Y2 = F.Y2[i];
    const double Y = Y1 + Y2;
    const double a = F.a0 * cos(t), da = -F.a0 * sin(t);
    const double z = F.c + a * Y;
    const double us = (double)theta + log(z / (1.0 - z)) / (double)beta;
    const double dus = da * Y / ((double)beta * z * (1.0 - z));
    return dus + us - (F.lam0 * F.c + a * (F.lam1 * Y1 + F.lam2 * Y2));
}

__global__ void rk4_stage_kernel(StageKArgs a) {
    const long long step = *a.step_ctr;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < (int64_t)a.B * a.n) {
        const int b = (int)(idx / a.n);
        const int64_t i = idx - (int64_t)b * a.n;
        float I = 0.f;
        for (int sp = 0; sp < a.splits; ++sp) I += a.partial[((int64_t)sp * a.B + b) * a.n_pad + i];
        if (a.rs) I *= a.rs[i];
        const double cs = (a.stage == 1) ? 0.0 : (a.stage == 4 ? 1.0 : 0.5);
        const double ts = *a.t0 + (double)step * a.dt + cs * a.dt;
        const float bb = a.beta[b], th = a.theta[b];
        const float gam = (float)forcing_value(a.F, i, ts, bb, th);
        const float Uv = a.U[idx], uv = a.u[idx];
        const float k = (-Uv + I) + gam;
        const float dt = (float)a.dt;
        float Un;
        if (a.stage == 1) {
            a.ks[idx] = k;
            Un = fmaf(0.5f * dt, k, uv);
        } else if (a.stage == 2) {
            a.ks[idx] = fmaf(2.f, k, a.ks[idx]);
            Un = fmaf(0.5f * dt, k, uv);
        } else if (a.stage == 3) {
            a.ks[idx] = fmaf(2.f, k, a.ks[idx]);
            Un = fmaf(dt, k, uv);
        } else {
            const float unew = fmaf(dt / 6.f, a.ks[idx] + k, uv);
            a.u[idx] = unew;
            Un = unew;
            if (a.ckpt && ((step + 1) % a.C) == 0)
                a.ckpt[(int64_t)((step + 1) / a.C) * a.B * a.n + idx] = unew;
        }
        a.U[idx] = Un;
        const float f = firing_rate(Un, bb, th);
        a.g[(int64_t)b * a.n_pad + i] = a.q ? a.q[i] * f : f;
    }
    if (a.stage == 4) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(a.done_ctr, 1u);
            if (prev == gridDim.x - 1) {
                *a.done_ctr = 0u;
                atomicAdd(reinterpret_cast<unsigned long long *>(a.step_ctr), 1ull);
                __threadfence();
            }
        }
    }
}

// Start a new nf_rk4_advance call: clock t0 and step counter 0.
__global__ void set_clock_kernel(double *t0_dev, long long *step_ctr, double t0) {
    *t0_dev = t0;
    *step_ctr = 0;
}

nf_status launch_set_clock(nf_operator *op, double t0, cudaStream_t s) {
    set_clock_kernel<<<1, 1, 0, s>>>(op->t0_dev, op->step_ctr, t0);
    NF_CUDA_TRY(cudaGetLastError());
    return NF_OK;
}

nf_status launch_stage(nf_operator *op, int B, const StageParams &p, cudaStream_t s) {
    StageKArgs a{};
    a.partial = op->partial;
    a.splits = p.splits;
    a.n = op->n;
    a.n_pad = op->n_pad;
    a.B = B;
    a.u = p.u;
    a.U = op->U;
    a.ks = op->ks;
    a.g = op->g;
    a.q = (op->path == NF_MATRIX_FREE) ? op->q : nullptr;
    a.rs = (op->path == NF_DENSE_BF16X2) ? op->rs : nullptr;
    a.beta = p.beta;
    a.theta = p.theta;
    a.F = p.forcing;
    a.t0 = op->t0_dev;
    a.dt = p.dt;
    a.stage = p.stage;
    a.step_ctr = op->step_ctr;
    a.done_ctr = op->done_ctr;
    a.ckpt = p.ckpt;
    a.C = p.C;
    const int64_t tot = (int64_t)B * op->n;
    const int T = 256;
    rk4_stage_kernel<<<(unsigned)ceil_div(tot, T), T, 0, s>>>(a);
    NF_CUDA_TRY(cudaGetLastError());
    return NF_OK;
}

}  // namespace nfi
