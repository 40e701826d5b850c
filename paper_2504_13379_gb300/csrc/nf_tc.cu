// nf_tc.cu -- batched path: several node sets ("groups"), each with B_g trajectories,
// advanced together with a grouped, persistent tcgen05 GEMM per RK4 stage.
//
// For group g with n_g nodes: D[i, b] = sum_j (Whi_ij Fhi_bj + Whi_ij Flo_bj + Wlo_ij Fhi_bj)
// (the bf16 x 3 split; the Wlo Flo term, ~2^-18 relative, is dropped), accumulated in FP32
// in tensor memory; I[b, i] = s_i D[i, b] with the operator's power-of-two row scales.  The
// epilogue of the GEMM is the RK4 stage of Eq. (2.9): k_s = -U_s + I_s, the tableau update,
// the next stage input and its firing rates f(U) split again into bf16 hi + lo, written
// K-major for the next stage's B operand (ping-pong buffers).
//
// Two-SM tiles.  CTAs run in clusters of two on neighbouring SMs; a pair owns 256 output rows
// and issues tcgen05.mma.cta_group::2 with M = 256: each CTA stages its own 128 rows of W hi/lo
// and one half of the F hi/lo tile (N/2 trajectory rows), which halves the L2 -> SM traffic
// for the shared F tile.  A pipeline stage covers K = 64 (128-byte rows, 128-byte swizzle):
// 32 KB of W and up to 32 KB of F per CTA, three stages deep.  Large stages matter more than
// deep rings here: each stage costs a fixed producer / consumer hand-off, and one SM streams
// about 100 GB/s with 64 KB stages against about 45 GB/s with 16 KB stages.
// 320 threads per CTA, one CTA per SM, persistent over a host-balanced list of pair tiles:
//   warp 0      TMA producer (both CTAs): W hi/lo tiles (128 x 64, one contiguous block of the
//               blocked layout each) and half F tiles (N/2 x 64); completion of both CTAs'
//               copies is counted on the leader CTA's "full" barrier
//   warp 1      owns the tensor-memory allocation (2 x 256 columns per CTA, double buffered);
//               in the leader CTA (rank 0) lane 0 issues the MMAs, N = B_g rounded to 16,
//               K = 16 per instruction, 3 products per K step, and commits to the "empty" and
//               "accumulator full" barriers of both CTAs (multicast)
//   warps 2..9  epilogue (both CTAs): two warps per TMEM lane quarter (one TMEM lane = one
//               row i), N/2 columns each; they drain the accumulator after every K chunk of
//               256, add it into FP32 registers and release the chunk buffer on the leader's
//               barrier; the fused RK4 stage update and next-stage bf16 split of a tile run
//               deferred, in slices between the next tile's chunk drains
// Chunking K matters for accuracy: the tensor core's FP32 accumulation truncates when
// aligning addends, an error that grows with the number of K steps summed in tensor
// memory; 256-wide chunks added with round-to-nearest FP32 adds keep the long sums
// (K up to 40,000 here) at the accuracy of the bf16 x 3 representation.
// Every wait on an mbarrier is bounded; on timeout the kernel records NF_ERR_TIMEOUT,
// stops issuing work, lets copies in flight land, frees its tensor memory and returns.
#include "nf_internal.cuh"

#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

namespace nfi {

constexpr int TC_M = 128;          // rows per CTA
constexpr int TC_PAIR_M = 256;     // rows per cluster pair (MMA M)
constexpr int TC_BK = 64;          // K elements per stage: 128-byte rows
constexpr int TC_NMAX = 256;      // trajectories of one sub-group (MMA N, tensor-memory columns)
constexpr int TC_STAGES = 3;      // ring slots in shared memory; a launch uses 2 or 3 (tuned)
constexpr int TC_MAXG = 8;        // sub-groups per launch: (node set, range of <= 256 trajectories)
constexpr int TC_MAXM = 8;        // node sets (member operators) of a grouped operator
constexpr int TC_THREADS = 320;    // warp 0 TMA, warp 1 TMEM + MMA, warps 2..9 epilogue
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_CHUNK = 4;        // K blocks (256 elements) accumulated in tensor memory per chunk
constexpr int TC_EPI_BATCH = 2;    // trajectory columns per batch of epilogue loads (accumulators live)
constexpr int TC_EPI_TAIL = 8;     // the same once the accumulators are written out

template <int V>
struct BatchTag {
    static constexpr int value = V;
};
constexpr uint32_t TC_A_BYTES = TC_M * TC_BK * 2;             // 16 KB per plane
constexpr uint32_t TC_BH_BYTES = (TC_NMAX / 2) * TC_BK * 2;   // 16 KB per plane: half of N = 256
constexpr uint32_t TC_STAGE_BYTES = 2 * TC_A_BYTES + 2 * TC_BH_BYTES;
constexpr size_t TC_SMEM = (size_t)TC_STAGES * TC_STAGE_BYTES + 1024;

// One sub-group: the rows of one member node set against a range of its trajectories.
struct TcGroup {
    int n, B, n_mma, mtiles;  // B: trajectories of the range; mtiles: pair tiles of 256 rows
    int nkb_pad;              // 32-column blocks per row block of the blocked W planes
    int64_t ldF;          // leading dimension (elements) of the F planes, [b][ldF]
    int64_t state_off;    // offset of the group's B x n block in the concatenated state
    int traj_off;         // offset of the group's trajectories in beta / theta
    const float *rs;
    uint16_t *Fhi_out, *Flo_out;
};

struct TcParams {
    CUtensorMap tmA_hi[TC_MAXG], tmA_lo[TC_MAXG], tmB_hi[TC_MAXG], tmB_lo[TC_MAXG];
    TcGroup grp[TC_MAXG];
    int ngroups;           // sub-groups
    int nst;               // ring slots in use (2 or 3)
    int tile_start[TC_MAXG + 1];
    const int *sched;      // pair tiles in processing order, cluster c owns sched[sched_off[c] ..]
    const int *sched_off;  // [clusters + 1]
    int mode;             // 0: write I, 1: RK4 stage
    float *I;             // mode 0 output (concatenated B_g x n_g blocks)
    float *Iscr;          // RK4 stages: nonlocal sums awaiting the deferred stage update
    float *u, *U, *ks;
    const float *beta, *theta;
    const double *t0;
    double dt;
    int stage;
    long long *step_ctr;
    unsigned *done_ctr;
    float *ckpt;
    int C;
    int64_t state_total;
    int *err;
};

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared-cluster address of this CTA's shared variable `p` as seen in cluster CTA `rank`.
__device__ __forceinline__ uint32_t mapa_u32(const void *p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}

// 2-D tiled load into this CTA's shared memory; the transaction bytes are counted on the
// barrier at shared-cluster address `bar` (the leader CTA's barrier, for both CTAs).
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// K-major operand, 128-byte swizzle: 8-row x 128-byte atoms stacked every 1024 bytes.
__device__ __forceinline__ uint64_t sdesc_sw128(const void *p) {
    const uint64_t a = smem_u32(p);
    return ((a & 0x3FFFFull) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void umma_bf16_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Arrive (once) on the barrier at the same shared-memory offset in both CTAs of the pair
// when all previously issued MMAs of this thread have completed.
__device__ __forceinline__ void umma_commit_pair(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Arrive on a barrier in another CTA of the cluster (shared-cluster address).  Default
// semantics (release at CTA scope): what must be ordered before it are this warp's tensor
// memory reads, which tcgen05.fence::before_thread_sync does; a cluster-scope release would
// also wait for the epilogue's outstanding global stores.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
        "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ int tile_group(const TcParams &p, int t) {
    int g = 0;
    while (g + 1 < p.ngroups && t >= p.tile_start[g + 1]) ++g;
    return g;
}

__device__ __forceinline__ float tc_firing(float u, float beta, float theta) {
    return 1.0f / (1.0f + expf(-beta * (u - theta)));
}

// Registers: the ten warps of a CTA sit three to a scheduler on two of the SM's four
// schedulers, and each scheduler's register file holds 16,384, so a thread may use at most
// 168 (a cap of 200 leaves no CTA resident); at 168 the epilogue's 128 FP32 accumulators
// spill about 130 bytes a thread.
template <int STAGE>  // 0: write I (nonlocal apply); 1..4: fused RK4 stage
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(TC_THREADS, 1)
    tc_grouped_kernel(const __grid_constant__ TcParams p) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES], accf[2], acce[2];
    __shared__ uint32_t tmem_base_sh;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const int cluster = (int)(blockIdx.x >> 1);
    const int tbeg = p.sched_off[cluster], tend = p.sched_off[cluster + 1];
    const long long step = *p.step_ctr;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);   // leader: one expect_tx arrival; both CTAs' bytes
            mbar_init(&empty[s], 1);  // multicast MMA commit
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);                   // multicast MMA commit
            mbar_init(&acce[b], 2 * TC_EPI_WARPS);    // leader: one arrival per epilogue warp of the pair
        }
        mbar_fence_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(2 * TC_NMAX));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();  // barriers of both CTAs initialised before any remote arrival
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    auto sA_hi = [&](int s) { return smem + (size_t)s * TC_STAGE_BYTES; };
    auto sA_lo = [&](int s) { return smem + (size_t)s * TC_STAGE_BYTES + TC_A_BYTES; };
    auto sB_hi = [&](int s) { return smem + (size_t)s * TC_STAGE_BYTES + 2 * TC_A_BYTES; };
    auto sB_lo = [&](int s) { return smem + (size_t)s * TC_STAGE_BYTES + 2 * TC_A_BYTES + TC_BH_BYTES; };
    bool timed_out = false;

    if (warp == 0) {
        // ------------------------------------------------------------- TMA producer
        if (lane == 0) {
            int s = 0;          // ring slot and its phase, advanced per K block
            uint32_t ph = 0;
            for (int ti = tbeg; ti < tend && !timed_out; ++ti) {
                const int t = p.sched[ti];
                const int g = tile_group(p, t);
                const TcGroup &G = p.grp[g];
                const int row0 = (t - p.tile_start[g]) * TC_PAIR_M + (int)rank * TC_M;
                const int nk = (G.n + TC_BK - 1) / TC_BK;
                const int nh = G.n_mma >> 1;
                const uint32_t bytes = 2 * (2 * TC_A_BYTES + 2u * (uint32_t)nh * TC_BK * 2u);
                for (int kb = 0; kb < nk; ++kb) {
                    if (!mbar_spin_bounded(&empty[s], ph ^ 1u)) {
                        timed_out = true;
                        break;
                    }
                    if (rank == 0) mbar_arrive_expect_tx(&full[s], bytes);
                    const uint32_t fb = mapa_u32(&full[s], 0);
                    const int wy = ((row0 >> 7) * G.nkb_pad + kb) * TC_M;  // block (row0 / 128, kb)
                    tma_load_2d_pair(sA_hi(s), &p.tmA_hi[g], 0, wy, fb);
                    tma_load_2d_pair(sA_lo(s), &p.tmA_lo[g], 0, wy, fb);
                    tma_load_2d_pair(sB_hi(s), &p.tmB_hi[g], kb * TC_BK, (int)rank * nh, fb);
                    tma_load_2d_pair(sB_lo(s), &p.tmB_lo[g], kb * TC_BK, (int)rank * nh, fb);
                    if (++s == p.nst) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (timed_out) set_dev_error(p.err, DEV_TIMEOUT);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------- MMA issuer (leader)
        if (lane == 0 && rank == 0) {
            uint32_t ci = 0;
            int s = 0;          // ring slot and its phase, as in the producer
            uint32_t ph = 0;
            for (int ti = tbeg; ti < tend && !timed_out; ++ti) {
                const int t = p.sched[ti];
                const int g = tile_group(p, t);
                const TcGroup &G = p.grp[g];
                const int nk = (G.n + TC_BK - 1) / TC_BK;
                const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(G.n_mma >> 3) << 17) |
                                       ((uint32_t)(TC_PAIR_M >> 4) << 24);
                // K is accumulated in tensor memory one chunk at a time; the epilogue adds
                // the chunks in FP32 registers (round to nearest)
                for (int kc = 0; kc < nk && !timed_out; kc += TC_CHUNK, ++ci) {
                    const uint32_t ab = ci & 1u, aph = (ci >> 1) & 1u;
                    if (!mbar_spin_bounded(&acce[ab], aph ^ 1u)) {
                        timed_out = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + ab * TC_NMAX;
                    const int kend = min(nk, kc + TC_CHUNK);
                    for (int kb = kc; kb < kend; ++kb) {
                        if (!mbar_spin_bounded(&full[s], ph)) {
                            timed_out = true;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t ahi = sdesc_sw128(sA_hi(s)), alo = sdesc_sw128(sA_lo(s));
                        const uint64_t bhi = sdesc_sw128(sB_hi(s)), blo = sdesc_sw128(sB_lo(s));
#pragma unroll
                        for (int k = 0; k < TC_BK / 16; ++k) {
                            const uint64_t off = (uint64_t)((k * 32) >> 4);
                            umma_bf16_pair(d, ahi + off, bhi + off, idesc, ((kb - kc) | k) ? 1u : 0u);
                            umma_bf16_pair(d, ahi + off, blo + off, idesc, 1u);
                            umma_bf16_pair(d, alo + off, bhi + off, idesc, 1u);
                        }
                        umma_commit_pair(&empty[s]);  // the slot is free in both CTAs once read
                        if (++s == p.nst) {
                            s = 0;
                            ph ^= 1u;
                        }
                    }
                    if (timed_out) break;
                    umma_commit_pair(&accf[ab]);      // chunk accumulators ready in both CTAs
                }
            }
            if (timed_out) set_dev_error(p.err, DEV_TIMEOUT);
        }
    } else {
        // ------------------------------------------------------------- epilogue
        // Two warps per TMEM lane quarter (warp & 3 selects the quarter a warp may
        // access); each owns half of the tile's N accumulator columns (at most 128).
        const int q4 = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row_in_tile = (int)rank * TC_M + 32 * q4 + lane;
        const uint32_t acce_leader[2] = {mapa_u32(&acce[0], 0), mapa_u32(&acce[1], 0)};
        uint32_t ci = 0;
        const float dtf = (float)p.dt;
        // Deferred RK4 update.  After its last chunk a tile's scaled sums go to the scratch
        // state Iscr and the warps move on to the next tile; the previous tile's stage update
        // runs in slices in the gaps between the next tile's chunk drains, so the tensor core
        // does not wait for its global-memory latency.  Pending job: group pg (< 0: none),
        // pair tile pmt, next column pnext (warp-uniform).
        int pg = -1, pmt = 0, pnext = 0;
        // NBT columns per batch of loads: TC_EPI_BATCH between chunk drains, while the 128
        // accumulators are live; TC_EPI_TAIL once they are written out (the rest of a tile and
        // the cluster's last tile, which no MMA overlaps), for more loads in flight.
        auto rk4_slice = [&](int upto, auto nbt_tag) {
            constexpr int NBT = decltype(nbt_tag)::value;
            if (pg < 0) return;
            const TcGroup &PG = p.grp[pg];
            const int pncol = PG.n_mma >> 1, pcol0 = half * pncol;
            const int end = min(upto, pncol);
            const int i = pmt * TC_PAIR_M + row_in_tile;
            if (i < PG.n) {
                const int64_t base = PG.state_off + i;
                for (int c0 = pnext; c0 < end && pcol0 + c0 < PG.B; c0 += NBT) {
                    // every load of the batch is issued before any result is used
                    float Dv[NBT], Uv[NBT], uv[NBT], kv[NBT], bb[NBT], th[NBT];
#pragma unroll
                    for (int j = 0; j < NBT; ++j) {
                        const int b = min(pcol0 + c0 + j, PG.B - 1);
                        const int64_t idx = base + (int64_t)b * PG.n;
                        Dv[j] = p.Iscr[idx];
                        Uv[j] = p.U[idx];
                        uv[j] = p.u[idx];
                        kv[j] = (STAGE > 1) ? p.ks[idx] : 0.f;
                        bb[j] = __ldg(p.beta + PG.traj_off + b);
                        th[j] = __ldg(p.theta + PG.traj_off + b);
                    }
#pragma unroll
                    for (int j = 0; j < NBT; ++j) {
                        const int b = pcol0 + c0 + j;
                        if (b >= PG.B || c0 + j >= end) break;
                        const int64_t idx = base + (int64_t)b * PG.n;
                        const float k = -Uv[j] + Dv[j];
                        float Un;
                        if constexpr (STAGE == 1) {
                            p.ks[idx] = k;
                            Un = fmaf(0.5f * dtf, k, uv[j]);
                        } else if constexpr (STAGE == 2) {
                            p.ks[idx] = fmaf(2.f, k, kv[j]);
                            Un = fmaf(0.5f * dtf, k, uv[j]);
                        } else if constexpr (STAGE == 3) {
                            p.ks[idx] = fmaf(2.f, k, kv[j]);
                            Un = fmaf(dtf, k, uv[j]);
                        } else {
                            Un = fmaf(dtf / 6.f, kv[j] + k, uv[j]);
                            p.u[idx] = Un;
                            if (p.ckpt && ((step + 1) % p.C) == 0)
                                p.ckpt[(int64_t)((step + 1) / p.C) * p.state_total + idx] = Un;
                        }
                        p.U[idx] = Un;
                        const float f = tc_firing(Un, bb[j], th[j]);
                        const __nv_bfloat16 hi = __float2bfloat16_rn(f);
                        const __nv_bfloat16 lo = __float2bfloat16_rn(f - __bfloat162float(hi));
                        PG.Fhi_out[(int64_t)b * PG.ldF + i] = __bfloat16_as_ushort(hi);
                        PG.Flo_out[(int64_t)b * PG.ldF + i] = __bfloat16_as_ushort(lo);
                    }
                }
            }
            pnext = end;
            if (pnext >= pncol) pg = -1;
        };
        for (int ti = tbeg; ti < tend && !timed_out; ++ti) {
            const int t = p.sched[ti];
            const int g = tile_group(p, t);
            const TcGroup &G = p.grp[g];
            const int mt = t - p.tile_start[g];
            const int nk = (G.n + TC_BK - 1) / TC_BK;
            const int ncol = G.n_mma >> 1;
            const int col0 = half * ncol;
            // columns of the pending job per chunk of this tile (whole batches)
            const int nchunks = (nk + TC_CHUNK - 1) / TC_CHUNK;
            const int pend = pg >= 0 ? (p.grp[pg].n_mma >> 1) - pnext : 0;
            const int per = ((pend + nchunks - 1) / nchunks + TC_EPI_BATCH - 1) / TC_EPI_BATCH * TC_EPI_BATCH;
            float acc[128];
#pragma unroll
            for (int c = 0; c < 128; ++c) acc[c] = 0.f;
            for (int kc = 0; kc < nk; kc += TC_CHUNK, ++ci) {
                const uint32_t ab = ci & 1u, aph = (ci >> 1) & 1u;
                if (STAGE > 0) rk4_slice(pnext + per, BatchTag<TC_EPI_BATCH>{});  // while this chunk is on the tensor core
                if (!mbar_wait_bounded(&accf[ab], aph)) {
                    if (lane == 0) set_dev_error(p.err, DEV_TIMEOUT);
                    timed_out = true;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (32 * c < ncol) {  // warp-uniform
                        uint32_t r[32];
                        tmem_ld32(tmem + ((uint32_t)(32 * q4) << 16) + ab * TC_NMAX + (uint32_t)(col0 + 32 * c), r);
#pragma unroll
                        for (int j = 0; j < 32; ++j) acc[32 * c + j] += __uint_as_float(r[j]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_remote(acce_leader[ab]);
            }
            if (timed_out) break;
            const int i = mt * TC_PAIR_M + row_in_tile;
            if (i < G.n) {
                const float si = G.rs[i];
                float *dst = STAGE == 0 ? p.I : p.Iscr;
                const int64_t base = G.state_off + i;
#pragma unroll
                for (int c = 0; c < 128; ++c) {
                    const int b = col0 + c;
                    if (c >= ncol || b >= G.B) break;
                    dst[base + (int64_t)b * G.n] = si * acc[c];
                }
            }
            if (STAGE > 0) {
                // whatever of the previous tile is left (other tiles' state than this one's)
                rk4_slice(1 << 30, BatchTag<TC_EPI_TAIL>{});
                pg = g;
                pmt = mt;
                pnext = 0;
            }
        }
        if (STAGE > 0 && !timed_out) rk4_slice(1 << 30, BatchTag<TC_EPI_TAIL>{});
    }
    // After a timeout, copies already issued may still land in shared memory and count on
    // the leader's barriers: give them time before the pair leaves (bounded, ~1 ms).
    if (__syncthreads_or(timed_out ? 1 : 0))
        for (int w = 0; w < 1000; ++w) __nanosleep(1000);
    tc_fence_before();
    cluster_sync();  // neither CTA leaves while the pair's MMAs or arrivals may touch it
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_NMAX));
    }
    if (STAGE == 4 && threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(p.done_ctr, 1u);
        if (prev == gridDim.x - 1) {
            *p.done_ctr = 0u;
            atomicAdd(reinterpret_cast<unsigned long long *>(p.step_ctr), 1ull);
            __threadfence();
        }
    }
}

// F planes for all groups from u: hi/lo split of f(u); optionally U = u.
struct TcPrepGroup {
    int n, B;
    int64_t ldF, state_off;
    int traj_off;
    uint16_t *Fhi, *Flo;
};
struct TcPrepArgs {
    TcPrepGroup grp[TC_MAXM];
    int ngroups;
    const float *u;
    float *U;
    const float *beta, *theta;
    int64_t total;
};

__global__ void tc_prep_kernel(TcPrepArgs a) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.total) return;
    int g = 0;
    while (g + 1 < a.ngroups && idx >= a.grp[g + 1].state_off) ++g;
    const TcPrepGroup &G = a.grp[g];
    const int64_t loc = idx - G.state_off;
    const int b = (int)(loc / G.n);
    const int64_t i = loc - (int64_t)b * G.n;
    const float uv = a.u[idx];
    const int tb = G.traj_off + b;
    const float f = tc_firing(uv, a.beta[tb], a.theta[tb]);
    const __nv_bfloat16 hi = __float2bfloat16_rn(f);
    const __nv_bfloat16 lo = __float2bfloat16_rn(f - __bfloat162float(hi));
    G.Fhi[(int64_t)b * G.ldF + i] = __bfloat16_as_ushort(hi);
    G.Flo[(int64_t)b * G.ldF + i] = __bfloat16_as_ushort(lo);
    if (a.U) a.U[idx] = uv;
}

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static nf_status encode_fn(EncodeTiledFn *out) {
    static std::mutex mu;
    static EncodeTiledFn fn = nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q{};
        NF_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q));
        if (!ptr || q != cudaDriverEntryPointSuccess) return fail(NF_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        fn = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    *out = fn;
    return NF_OK;
}

// 2-D bf16 map over a row-major [rows][ld] plane, extent (cols x rows), box (TC_BK x box_rows).
static nf_status make_map(CUtensorMap *m, const void *base, int64_t cols, int64_t rows, int64_t ld, int box_rows) {
    EncodeTiledFn enc = nullptr;
    NF_TRY(encode_fn(&enc));
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    const cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(NF_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return NF_OK;
}

}  // namespace nfi

// Group state lives in the grouped operator handle.
struct nf_group_state {
    int count = 0;                           // member node sets
    nf_operator *members[nfi::TC_MAXM] = {};
    int B[nfi::TC_MAXM] = {};
    int64_t state_off[nfi::TC_MAXM] = {};    // member blocks in the concatenated state (caller order)
    int traj_off[nfi::TC_MAXM] = {};
    uint16_t *F[nfi::TC_MAXM][2][2] = {};    // [member][buffer][hi/lo]: B_m x n_pad bf16 planes
    // sub-groups in launch order (most trajectories first): member, first trajectory, count
    int nsub = 0;
    int sub_m[nfi::TC_MAXG] = {}, sub_b0[nfi::TC_MAXG] = {}, sub_nb[nfi::TC_MAXG] = {};
    int64_t state_total = 0;
    int traj_total = 0;
    int nclusters = 0;                       // CTA pairs per launch
    float *Iscr = nullptr;                   // state_total: sums awaiting the deferred RK4 update
    int *sched = nullptr;                    // device: [nclusters + 1] offsets, then the tile list
    nfi::TcParams params[2];                 // [0]: reads F buffer 0, writes 1; [1]: reads 1, writes 0
    // launch configuration chosen by the autotuner at nf_operator_group
    int nst = nfi::TC_STAGES;                // ring slots in use
    int split = 1;                           // pieces a member of >= 128 trajectories is cut into
    double lpt_coef = 8.0;                   // MMA weight of a tile's K step in the LPT cost
    float tuned_ms = 0.f;                    // the chosen configuration's time per launch
};

namespace nfi {

// Cut every member's trajectories into sub-groups of at most TC_NMAX: ceil(B / 256) pieces,
// or `split` pieces for members of at least 128 trajectories when that is more; piece sizes
// are multiples of 16 (the MMA's N granularity) except the last.  Launch order: most
// trajectories first.  Returns false when the pieces exceed TC_MAXG.
static bool make_subgroups(nf_group_state *gs, int split) {
    int m_of[TC_MAXG * 4], b0_of[TC_MAXG * 4], nb_of[TC_MAXG * 4];
    int cnt = 0;
    for (int m = 0; m < gs->count; ++m) {
        const int Bm = gs->B[m];
        int np = (Bm + TC_NMAX - 1) / TC_NMAX;
        if (Bm >= 128) np = std::max(np, split);
        const int piece = ((Bm + np - 1) / np + 15) / 16 * 16;
        for (int b0 = 0; b0 < Bm; b0 += piece) {
            if (cnt == TC_MAXG) return false;
            m_of[cnt] = m;
            b0_of[cnt] = b0;
            nb_of[cnt] = std::min(piece, Bm - b0);
            ++cnt;
        }
    }
    int order[TC_MAXG];
    std::iota(order, order + cnt, 0);
    std::stable_sort(order, order + cnt, [&](int a, int b) { return nb_of[a] > nb_of[b]; });
    gs->nsub = cnt;
    for (int k = 0; k < cnt; ++k) {
        gs->sub_m[k] = m_of[order[k]];
        gs->sub_b0[k] = b0_of[order[k]];
        gs->sub_nb[k] = nb_of[order[k]];
    }
    return true;
}

static nf_status build_group_params(nf_operator *op) {
    nf_group_state *gs = op->group;
    for (int par = 0; par < 2; ++par) {
        TcParams &P = gs->params[par];
        memset(&P, 0, sizeof(P));
        P.ngroups = gs->nsub;
        P.nst = gs->nst;
        int tiles = 0;
        for (int k = 0; k < gs->nsub; ++k) {
            const int m = gs->sub_m[k], b0 = gs->sub_b0[k];
            nf_operator *mo = gs->members[m];
            TcGroup &G = P.grp[k];
            G.n = (int)mo->n;
            G.B = gs->sub_nb[k];
            G.n_mma = (G.B + 15) / 16 * 16;
            G.mtiles = (int)ceil_div(mo->n, TC_PAIR_M);
            G.ldF = mo->n_pad;
            G.state_off = gs->state_off[m] + (int64_t)b0 * mo->n;
            G.traj_off = gs->traj_off[m] + b0;
            G.rs = mo->rs;
            const int in = par, out = 1 - par;
            const int64_t foff = (int64_t)b0 * mo->n_pad;  // 16-byte aligned: n_pad is a multiple of 1024
            G.Fhi_out = gs->F[m][out][0] + foff;
            G.Flo_out = gs->F[m][out][1] + foff;
            // W planes in the blocked layout: viewed as (n_pad / 128) x (n_pad / 64) blocks of
            // 128 rows x 64 columns stacked row after row, so block (rb, kb) starts at row
            // (rb * n_pad / 64 + kb) * 128 of a 64-column matrix
            const int64_t wrows = mo->n_pad * (mo->n_pad / kBlkCols);
            NF_TRY(make_map(&P.tmA_hi[k], mo->Whi, kBlkCols, wrows, kBlkCols, TC_M));
            NF_TRY(make_map(&P.tmA_lo[k], mo->Wlo, kBlkCols, wrows, kBlkCols, TC_M));
            G.nkb_pad = (int)(mo->n_pad / kBlkCols);
            // each CTA of a pair stages half of the sub-group's N trajectory rows
            NF_TRY(make_map(&P.tmB_hi[k], gs->F[m][in][0] + foff, mo->n, G.B, mo->n_pad, G.n_mma / 2));
            NF_TRY(make_map(&P.tmB_lo[k], gs->F[m][in][1] + foff, mo->n, G.B, mo->n_pad, G.n_mma / 2));
            P.tile_start[k] = tiles;
            tiles += G.mtiles;
        }
        P.tile_start[gs->nsub] = tiles;
        P.state_total = gs->state_total;
        P.err = op->err;
        P.step_ctr = op->step_ctr;
        P.done_ctr = op->done_ctr;
        P.t0 = op->t0_dev;
    }
    return NF_OK;
}

// Longest-processing-time assignment of the pair tiles to the clusters of one launch.  A
// tile's cost is its number of 32-wide K steps times the larger of an MMA term, coef x N
// (N = the sub-group's MMA width; the tensor-core time of a step grows with N), and a
// floor of 840 for streaming its 16 KB of W hi/lo at an even share of HBM bandwidth; coef
// is chosen by the autotuner.  Every other cluster runs its list backwards, so that wide
// (tensor-bound) and narrow (HBM-bound) tiles overlap instead of running in two phases.
static nf_status build_schedule(nf_operator *op, double coef, cudaStream_t s) {
    nf_group_state *gs = op->group;
    const TcParams &P = gs->params[0];
    const int ntiles = P.tile_start[P.ngroups];
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(num_sms() & ~1), 1, 1);
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = TC_SMEM;
    int maxc = 0;
    NF_CUDA_TRY(cudaOccupancyMaxActiveClusters(&maxc, tc_grouped_kernel<1>, &cfg));
    if (maxc < 1) return fail(NF_ERR_UNSUPPORTED, "no CTA pair of the batched GEMM fits on this device");
    const int nclust = std::min(ntiles, maxc);
    std::vector<double> cost(ntiles);
    for (int k = 0; k < P.ngroups; ++k) {
        const TcGroup &G = P.grp[k];
        const double c = (double)ceil_div(G.n, 32) * std::max(coef * G.n_mma, 840.0);
        for (int t = P.tile_start[k]; t < P.tile_start[k + 1]; ++t) cost[t] = c;
    }
    std::vector<int> order(ntiles);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> load(nclust, 0.0);
    std::vector<std::vector<int>> lists(nclust);
    for (int t : order) {
        const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lists[c].push_back(t);
        load[c] += cost[t];
    }
    for (int c = 1; c < nclust; c += 2) std::reverse(lists[c].begin(), lists[c].end());
    std::vector<int> host;
    host.reserve(nclust + 1 + ntiles);
    int off = 0;
    for (int c = 0; c < nclust; ++c) {
        host.push_back(off);
        off += (int)lists[c].size();
    }
    host.push_back(off);
    for (int c = 0; c < nclust; ++c) host.insert(host.end(), lists[c].begin(), lists[c].end());
    NF_CUDA_TRY(cudaStreamSynchronize(s));  // no launch may still read the previous list
    if (gs->sched) NF_CUDA_TRY(cudaFree(gs->sched));
    gs->sched = nullptr;
    NF_CUDA_TRY(cudaMalloc(&gs->sched, sizeof(int) * host.size()));
    NF_CUDA_TRY(cudaMemcpyAsync(gs->sched, host.data(), sizeof(int) * host.size(), cudaMemcpyHostToDevice, s));
    NF_CUDA_TRY(cudaStreamSynchronize(s));
    gs->nclusters = nclust;
    for (int par = 0; par < 2; ++par) {
        gs->params[par].sched_off = gs->sched;
        gs->params[par].sched = gs->sched + nclust + 1;
    }
    return NF_OK;
}

void destroy_group(nf_operator *op) {
    if (!op->group) return;
    nf_group_state *gs = op->group;
    cudaFree(gs->sched);
    cudaFree(gs->Iscr);
    for (int m = 0; m < gs->count; ++m)
        for (int b = 0; b < 2; ++b)
            for (int h = 0; h < 2; ++h) cudaFree(gs->F[m][b][h]);
    delete gs;
    op->group = nullptr;
}

int group_traj_total(const nf_operator *op) { return op->group ? op->group->traj_total : 0; }
int64_t group_state_total(const nf_operator *op) { return op->group ? op->group->state_total : 0; }

nf_status tc_prep(nf_operator *op, const float *u, const float *beta, const float *theta, bool copy_U, int buffer,
                  cudaStream_t s) {
    nf_group_state *gs = op->group;
    TcPrepArgs a{};
    a.ngroups = gs->count;
    for (int m = 0; m < gs->count; ++m) {
        TcPrepGroup &G = a.grp[m];
        G.n = (int)gs->members[m]->n;
        G.B = gs->B[m];
        G.ldF = gs->members[m]->n_pad;
        G.state_off = gs->state_off[m];
        G.traj_off = gs->traj_off[m];
        G.Fhi = gs->F[m][buffer][0];
        G.Flo = gs->F[m][buffer][1];
    }
    a.u = u;
    a.U = copy_U ? op->U : nullptr;
    a.beta = beta;
    a.theta = theta;
    a.total = gs->state_total;
    tc_prep_kernel<<<(unsigned)ceil_div(a.total, 256), 256, 0, s>>>(a);
    NF_CUDA_TRY(cudaGetLastError());
    return NF_OK;
}

nf_status tc_launch(nf_operator *op, int parity, int mode, float *I, float *u, const float *beta, const float *theta,
                    double dt, int stage, float *ckpt, int C, cudaStream_t s) {
    TcParams P = op->group->params[parity];
    P.mode = mode;
    P.I = I;
    P.Iscr = op->group->Iscr;
    P.u = u;
    P.U = op->U;
    P.ks = op->ks;
    P.beta = beta;
    P.theta = theta;
    P.dt = dt;
    P.stage = stage;
    P.ckpt = ckpt;
    P.C = C;
    const int grid = 2 * op->group->nclusters;
    switch (mode == 0 ? 0 : stage) {
        case 0: tc_grouped_kernel<0><<<grid, TC_THREADS, TC_SMEM, s>>>(P); break;
        case 1: tc_grouped_kernel<1><<<grid, TC_THREADS, TC_SMEM, s>>>(P); break;
        case 2: tc_grouped_kernel<2><<<grid, TC_THREADS, TC_SMEM, s>>>(P); break;
        case 3: tc_grouped_kernel<3><<<grid, TC_THREADS, TC_SMEM, s>>>(P); break;
        default: tc_grouped_kernel<4><<<grid, TC_THREADS, TC_SMEM, s>>>(P); break;
    }
    NF_CUDA_TRY(cudaGetLastError());
    return NF_OK;
}

nf_status tc_init_attr() {
    NF_CUDA_TRY(cudaFuncSetAttribute(tc_grouped_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    NF_CUDA_TRY(cudaFuncSetAttribute(tc_grouped_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    NF_CUDA_TRY(cudaFuncSetAttribute(tc_grouped_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    NF_CUDA_TRY(cudaFuncSetAttribute(tc_grouped_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    NF_CUDA_TRY(cudaFuncSetAttribute(tc_grouped_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    return NF_OK;
}

}  // namespace nfi

using namespace nfi;

namespace nfi {

// Time one launch configuration: one warm-up and two timed nonlocal-sum launches (mode 0,
// output into the group's scratch state); the faster timed launch counts.
static nf_status time_config(nf_operator *op, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float *ms) {
    nf_group_state *gs = op->group;
    float best = 3.4e38f;
    for (int rep = 0; rep < 3; ++rep) {
        NF_CUDA_TRY(cudaEventRecord(e0, s));
        NF_TRY(tc_launch(op, 0, 0, gs->Iscr, nullptr, nullptr, nullptr, 0.0, 0, nullptr, 1, s));
        NF_CUDA_TRY(cudaEventRecord(e1, s));
        NF_CUDA_TRY(cudaEventSynchronize(e1));
        float t = 0.f;
        NF_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
        if (rep > 0) best = std::min(best, t);
    }
    *ms = best;
    return NF_OK;
}

// The batched path's autotuner.  Candidates: trajectory split {1, 2} (a member of 128..256
// trajectories as one sub-group of MMA width up to 256, or as two of half the width: more
// tiles to balance, W streamed twice), LPT weight of the MMA term {4, 8, 12} (how much more
// a wide tile costs than a narrow, HBM-bound one), ring depth {3, 2} (64 KB slots in flight).
// Each candidate is timed on the device (time_config) and the fastest is kept; the results
// do not depend on the choice (each output is the same MMA chain over K in the same order).
static nf_status tc_autotune(nf_operator *op, cudaStream_t s) {
    nf_group_state *gs = op->group;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    NF_CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ce, "cudaEventCreate", __FILE__, __LINE__);
    }
    struct Best {
        int split, nst;
        double coef;
        float ms;
    } best{1, TC_STAGES, 8.0, 3.4e38f};
    nf_status st = NF_OK;
    const int splits[2] = {1, 2};
    const double coefs[3] = {4.0, 8.0, 12.0};
    const int depths[2] = {TC_STAGES, 2};
    for (int a = 0; a < 2 && st == NF_OK; ++a) {
        if (!make_subgroups(gs, splits[a])) continue;
        if (a > 0) {  // a split that changes nothing is not timed twice
            bool changed = false;
            for (int m = 0; m < gs->count; ++m) changed |= gs->B[m] >= 128;
            if (!changed) continue;
        }
        for (int c = 0; c < 3 && st == NF_OK; ++c) {
            for (int d = 0; d < 2 && st == NF_OK; ++d) {
                gs->nst = depths[d];
                st = build_group_params(op);
                if (st == NF_OK) st = build_schedule(op, coefs[c], s);
                float ms = 0.f;
                if (st == NF_OK) st = time_config(op, s, e0, e1, &ms);
                if (st == NF_OK && ms < best.ms) best = Best{splits[a], depths[d], coefs[c], ms};
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != NF_OK) return st;
    gs->split = best.split;
    gs->nst = best.nst;
    gs->lpt_coef = best.coef;
    gs->tuned_ms = best.ms;
    if (!make_subgroups(gs, gs->split)) return fail(NF_ERR_UNSUPPORTED, "no feasible sub-group split");
    NF_TRY(build_group_params(op));
    return build_schedule(op, gs->lpt_coef, s);
}

}  // namespace nfi

extern "C" nf_status nf_operator_group(nf_operator *const *ops, const int *B_per_op, int count, void *stream,
                                       nf_operator **grouped) {
    clear_error();
    NF_ARG(ops && B_per_op && grouped, "ops, B_per_op and grouped must be non-NULL");
    *grouped = nullptr;
    NF_ARG(count >= 1 && count <= TC_MAXM, "count = %d must be in 1..%d", count, TC_MAXM);
    int pieces = 0;
    for (int m = 0; m < count; ++m) {
        NF_ARG(ops[m], "ops[%d] is NULL", m);
        NF_ARG(ops[m]->path == NF_DENSE_BF16X2, "ops[%d] must use the NF_DENSE_BF16X2 path", m);
        NF_ARG(B_per_op[m] >= 1 && B_per_op[m] <= TC_MAXG * TC_NMAX, "B[%d] = %d must be in 1..%d", m, B_per_op[m],
               TC_MAXG * TC_NMAX);
        NF_ARG(ops[m]->n >= TC_BK, "ops[%d] has n = %lld < %d nodes", m, (long long)ops[m]->n, TC_BK);
        pieces += (B_per_op[m] + TC_NMAX - 1) / TC_NMAX;
    }
    if (pieces > TC_MAXG)
        return fail(NF_ERR_UNSUPPORTED,
                    "the members need %d sub-groups of <= %d trajectories; one launch holds at most %d", pieces,
                    TC_NMAX, TC_MAXG);
    NF_TRY(tc_init_attr());
    cudaStream_t s = as_stream(stream);
    nf_operator *op = new nf_operator();
    op->path = NF_GROUPED;
    op->device = device_id();
    op->kp = ops[0]->kp;
    nf_group_state *gs = new nf_group_state();
    op->group = gs;
    gs->count = count;
    int64_t total = 0;
    int traj = 0;
    for (int m = 0; m < count; ++m) {
        gs->members[m] = ops[m];
        gs->B[m] = B_per_op[m];
        gs->state_off[m] = total;
        gs->traj_off[m] = traj;
        total += (int64_t)B_per_op[m] * ops[m]->n;
        traj += B_per_op[m];
    }
    gs->state_total = total;
    gs->traj_total = traj;
    op->n = total;  // state length of one "trajectory" of the group (the concatenation)
    op->n_pad = total;
    auto cleanup = [&](nf_status st) {
        nf_operator_destroy(op);
        return st;
    };
    for (int m = 0; m < count; ++m)
        for (int b = 0; b < 2; ++b)
            for (int h = 0; h < 2; ++h) {
                const size_t bytes = sizeof(uint16_t) * (size_t)B_per_op[m] * ops[m]->n_pad;
                cudaError_t e = cudaMalloc(&gs->F[m][b][h], bytes);
                if (e == cudaSuccess) e = cudaMemsetAsync(gs->F[m][b][h], 0, bytes, s);
                if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc(F)", __FILE__, __LINE__));
            }
    cudaError_t e = cudaMalloc(&op->step_ctr, 64);
    if (e == cudaSuccess) e = cudaMemsetAsync(op->step_ctr, 0, 64, s);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc(ctr)", __FILE__, __LINE__));
    op->done_ctr = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(op->step_ctr) + 16);
    op->err = reinterpret_cast<int *>(reinterpret_cast<char *>(op->step_ctr) + 32);
    op->t0_dev = reinterpret_cast<double *>(reinterpret_cast<char *>(op->step_ctr) + 40);
    e = cudaMalloc(&op->U, sizeof(float) * total);
    if (e == cudaSuccess) e = cudaMalloc(&op->ks, sizeof(float) * total);
    if (e == cudaSuccess) e = cudaMalloc(&gs->Iscr, sizeof(float) * total);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc(state)", __FILE__, __LINE__));
    op->state_cap = (size_t)total;
    nf_status st = tc_autotune(op, s);
    if (st == NF_OK) {  // the tuning launches may have recorded a timeout; start clean
        int flag = 0;
        e = cudaMemcpy(&flag, op->err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMemcpy(flag)", __FILE__, __LINE__);
        else if (flag != 0) st = fail(NF_ERR_TIMEOUT, "a bounded wait gave up while tuning the batched GEMM");
    }
    if (st != NF_OK) return cleanup(st);
    *grouped = op;
    return NF_OK;
}

extern "C" nf_status nf_operator_group_configure(nf_operator *op, int ring_depth, int traj_split, double lpt_coef,
                                                 void *stream) {
    clear_error();
    NF_ARG(op && op->path == NF_GROUPED && op->group, "not a grouped operator");
    NF_ARG(ring_depth == 2 || ring_depth == 3, "ring_depth = %d must be 2 or 3", ring_depth);
    NF_ARG(traj_split == 1 || traj_split == 2, "traj_split = %d must be 1 or 2", traj_split);
    NF_ARG(std::isfinite(lpt_coef) && lpt_coef > 0.0, "lpt_coef must be finite and > 0");
    nf_group_state *gs = op->group;
    cudaStream_t s = as_stream(stream);
    NF_CUDA_TRY(cudaStreamSynchronize(s));  // no launch may still use the current parameters
    if (!make_subgroups(gs, traj_split))
        return fail(NF_ERR_UNSUPPORTED, "traj_split = %d needs more than %d sub-groups", traj_split, TC_MAXG);
    destroy_graphs(op);  // captured steps hold the old parameters
    gs->split = traj_split;
    gs->nst = ring_depth;
    gs->lpt_coef = lpt_coef;
    gs->tuned_ms = 0.f;
    NF_TRY(build_group_params(op));
    return build_schedule(op, lpt_coef, s);
}

extern "C" nf_status nf_operator_group_tuning(nf_operator *op, int *ring_depth, int *traj_split, double *lpt_coef,
                                              int *subgroups, float *ms) {
    clear_error();
    NF_ARG(op && ring_depth && traj_split && lpt_coef && subgroups && ms, "arguments must be non-NULL");
    NF_ARG(op->path == NF_GROUPED && op->group, "not a grouped operator");
    const nf_group_state *gs = op->group;
    *ring_depth = gs->nst;
    *traj_split = gs->split;
    *lpt_coef = gs->lpt_coef;
    *subgroups = gs->nsub;
    *ms = gs->tuned_ms;
    return NF_OK;
}
