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
#include <atomic>
#include <cfloat>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

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
               int64_t jchunk, float c1, float c2, float A1, float A2, float per, float *__restrict__ partial,
               int *__restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const float iper = per > 0.f ? 1.f / per : 0.f;
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
        auto sweep = [&](auto tag) {
            constexpr bool P = decltype(tag)::value;
#pragma unroll 4
        for (int jj = lane; jj < MF_TJ; jj += 32) {
            const float4 xj = xs[jj];
            float gb[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) gb[b] = sm.gs[buf][b][jj];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float dx = xi[r] - xj.x, dy = yi[r] - xj.y;
                const float dz = zi[r] - xj.z;
                if constexpr (P) {
                    dx = wrap1(dx, per, iper);
                    dy = wrap1(dy, per, iper);
                }
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
        };
        if (per > 0.f)
            sweep(PerTag<true>{});
        else
            sweep(PerTag<false>{});
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
// duplicated in a 64-bit register pair.  Difference form, per two pairs: 3 SUB2, MUL2 +
// 2 FMA2 (r^2), MUL2 (second exponent), 4 MUFU.EX2, 2 FMA2 -- the rounding of the scalar
// kernel.  Expanded form (below): 3 FMA2, MUL2, 4 MUFU.EX2, 2 FMA2, plus 6 per column pair
// shared by the warp's rows, which leaves the SFU (2 exponentials per pair) as the bound.
typedef unsigned long long u64;
__device__ __forceinline__ u64 f2_sub(u64 a, u64 b) {
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 f2_add(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
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

// Nearest image of a packed pair of coordinate differences (see wrap1): ip = 1/p, np = -p,
// mg = the rounding constant, each in both halves.
__device__ __forceinline__ u64 f2_wrap(u64 d, u64 ip, u64 np, u64 mg) {
    return f2_fma(f2_sub(f2_fma(d, ip, mg), mg), np, d);
}

template <int TJ>
struct MfPackedSmem {
    float xs[2][TJ], ys[2][TJ], zs[2][TJ], gs[2][TJ];
    uint64_t bar[2];
};

// Rows are taken in a spatially coherent order (rowperm: Morton order of the nodes), so the
// R rows of a warp usually lie close together.  Such a warp expands the squared distance
// about the centre c of its rows' bounding box:
//   r^2 = |x_i - c|^2 + |x_j - c|^2 - 2 (x_i - c).(x_j - c) = n_i + s_ij,
//   s_ij = n_j - 2 (x_i - c).(x_j - c),
// and accumulates 2^(-s_ij) and 2^(-k2 s_ij); the row factors 2^(-n_i), 2^(-k2 n_i) are
// applied once at the end.  Per column pair the centred coordinates and n_j cost 6 lane
// operations shared by the warp's R rows; per pair the exponent argument is then a chain
// of 3 FMAs instead of 3 SUB + MUL + 2 FMA.  FP32 rounding of s_ij is relative to
// n_i + n_j + 2 |x_i - c||x_j - c|, so the form is used only when every row of the warp has
// n_i <= kMfLocalSpread (scaled units, i.e. |x_i - c| <= s1 / sqrt(log2 e)); for pairs
// that carry weight this keeps the error at a few ulps of r^2, the same order as the
// rounding of the stored coordinates.  Warps whose rows are spread out use the difference
// form.  The choice is warp-uniform and fixed per launch shape, so results stay
// deterministic.
//
// Integer width ratio.  When m = s2^2 / s1^2 is a small integer (M = 2, 3, 4; the paper's
// lateral-inhibition kernels have sigma_i = 2 sigma_e, i.e. m = 4), the expanded form works
// in units of s2 -- centred column coordinates times s1/s2 -- and takes e2 = 2^(-s'_ij)
// from the SFU and e1 = e2^M by squaring on the FMA pipe: one exponential per pair
// instead of two.  The relative error of e1 grows to about M times that of ex2.approx
// (a few 1e-7).  M = 0 is the general form.
constexpr float kMfLocalSpread = 1.0f;
// The symmetric kernel's threshold: rows within 2 s1 / sqrt(log2 e) of their centre.  The
// rounding of r^2 = n_i + s_ij for the pairs that carry weight stays of order eps * n_i
// (below 3e-7 relative in the exponential at n_i = 4); the expanded form saves three of the
// difference form's six exponent operations per pair.  Measured on GB300 against a threshold
// of 1: the same error against the FP64 oracle (1.4e-7 relative L2 on the precision torus,
// 9.3e-7 on the periodic square), 1.80 vs 1.82 ms on the precision torus, 2.37 vs 2.63 ms on
// the periodic square at n = 131,072, 0.157 vs 0.175 ms on the 20,000-node sphere.
constexpr float kSymLocalSpread = 4.0f;

// xyz: pre-scaled coordinates as structure of arrays [x(n_pad) | y(n_pad) | z(n_pad)],
// multiplied by sqrt(log2 e) / s1; g_all: B x n_pad firing rates (times q); rowperm: n_pad
// node indices, a permutation (padding rows map to themselves).
template <int R, int TJ, int M>
__global__ void __launch_bounds__(MF_THREADS, R >= 8 ? 2 : 4)
mf_pair_packed_kernel(const float *__restrict__ xyz, const float *__restrict__ g_all, const int *__restrict__ rowperm,
                      int64_t n_pad, int B, int b_base, int64_t jchunk, float k2, float A1, float A2,
                      float per, float *__restrict__ partial, int *__restrict__ err) {
    static_assert(M == 0 || (M >= 2 && M <= 4), "width ratio M must be 0 (general), 2, 3 or 4");
    __shared__ __align__(128) MfPackedSmem<TJ> sm;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int split = blockIdx.y;
    const int64_t j0 = (int64_t)split * jchunk;
    const int64_t j1 = min(n_pad, j0 + jchunk);
    const int ntiles = (int)((j1 - j0) / TJ);
    const int64_t slot0 = ((int64_t)blockIdx.x * MF_WARPS + warp) * R;
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
    // the warp's rows (all lanes hold the same values) and the centre of their bounding box
    float xr[R], yr[R], zr[R];
    float lox = 3.4e38f, loy = 3.4e38f, loz = 3.4e38f, hix = -3.4e38f, hiy = -3.4e38f, hiz = -3.4e38f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = __ldg(rowperm + slot0 + r);
        xr[r] = X[row];
        yr[r] = Y[row];
        zr[r] = Z[row];
        lox = fminf(lox, xr[r]), hix = fmaxf(hix, xr[r]);
        loy = fminf(loy, yr[r]), hiy = fmaxf(hiy, yr[r]);
        loz = fminf(loz, zr[r]), hiz = fmaxf(hiz, zr[r]);
    }
    const float cx = 0.5f * (lox + hix), cy = 0.5f * (loy + hiy), cz = 0.5f * (loz + hiz);
    float spread = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float dx = xr[r] - cx, dy = yr[r] - cy, dz = zr[r] - cz;
        spread = fmaxf(spread, dx * dx + dy * dy + dz * dz);
    }
    // warp-uniform; periodic distances take the difference form (nearest images per pair)
    const bool local = spread <= kMfLocalSpread && !(per > 0.f);
    // local: xi, yi, zi hold -2 (x_i - c) (times s1/s2 when M > 0); otherwise x_i itself
    // (both halves of the pair)
    const float sk = M > 0 ? sqrtf(k2) : 1.f;
    const float lsc = -2.f * sk;
    u64 xi[R], yi[R], zi[R], a1[R], a2[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float x = local ? lsc * (xr[r] - cx) : xr[r];
        const float y = local ? lsc * (yr[r] - cy) : yr[r];
        const float z = local ? lsc * (zr[r] - cz) : zr[r];
        xi[r] = f2_pack(x, x);
        yi[r] = f2_pack(y, y);
        zi[r] = f2_pack(z, z);
        a1[r] = 0ull;
        a2[r] = 0ull;
    }
    // coordinates arrive pre-scaled by sqrt(log2(e)) / s1, so r2s = r^2 log2(e) / s1^2:
    // e1 = 2^(-r2s), e2 = 2^(-k2 r2s) with k2 = s1^2 / s2^2
    const u64 nk2 = f2_pack(-k2, -k2);
    const u64 cxp = f2_pack(cx, cx), cyp = f2_pack(cy, cy), czp = f2_pack(cz, cz), skp = f2_pack(sk, sk);
    const float iper = per > 0.f ? 1.f / per : 0.f;
    const u64 ipp = f2_pack(iper, iper), npp = f2_pack(-per, -per), mgp = f2_pack(kRintMagic, kRintMagic);
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
        if (M > 0 && local) {
#pragma unroll 2
            for (int jp = lane; jp < TJ / 2; jp += 32) {
                const u64 xt = f2_mul(f2_sub(xs[jp], cxp), skp), yt = f2_mul(f2_sub(ys[jp], cyp), skp),
                          zt = f2_mul(f2_sub(zs[jp], czp), skp);
                const u64 nj = f2_fma(zt, zt, f2_fma(yt, yt, f2_mul(xt, xt)));
                const u64 gj = gs[jp];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const u64 sij = f2_fma(xi[r], xt, f2_fma(yi[r], yt, f2_fma(zi[r], zt, nj)));
                    float s0, s1v;
                    f2_unpack(sij, s0, s1v);
                    const u64 e2 = f2_pack(ex2_sfu(-s0), ex2_sfu(-s1v));
                    const u64 sq = f2_mul(e2, e2);
                    const u64 e1 = M == 2 ? sq : (M == 3 ? f2_mul(sq, e2) : f2_mul(sq, sq));
                    a1[r] = f2_fma(e1, gj, a1[r]);
                    a2[r] = f2_fma(e2, gj, a2[r]);
                }
            }
        } else if (local) {
#pragma unroll 2
            for (int jp = lane; jp < TJ / 2; jp += 32) {
                const u64 xt = f2_sub(xs[jp], cxp), yt = f2_sub(ys[jp], cyp), zt = f2_sub(zs[jp], czp);
                const u64 nj = f2_fma(zt, zt, f2_fma(yt, yt, f2_mul(xt, xt)));
                const u64 gj = gs[jp];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const u64 sij = f2_fma(xi[r], xt, f2_fma(yi[r], yt, f2_fma(zi[r], zt, nj)));
                    float s0, s1v;
                    f2_unpack(sij, s0, s1v);
                    const u64 e1 = f2_pack(ex2_sfu(-s0), ex2_sfu(-s1v));
                    const u64 e2 = f2_ex2(f2_mul(sij, nk2));
                    a1[r] = f2_fma(e1, gj, a1[r]);
                    a2[r] = f2_fma(e2, gj, a2[r]);
                }
            }
        } else {
            auto sweep = [&](auto tag) {
                constexpr bool P = decltype(tag)::value;
#pragma unroll 2
            for (int jp = lane; jp < TJ / 2; jp += 32) {
                const u64 xj = xs[jp], yj = ys[jp], zj = zs[jp], gj = gs[jp];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    u64 dx = f2_sub(xi[r], xj), dy = f2_sub(yi[r], yj);
                    const u64 dz = f2_sub(zi[r], zj);
                    if constexpr (P) {
                        dx = f2_wrap(dx, ipp, npp, mgp);
                        dy = f2_wrap(dy, ipp, npp, mgp);
                    }
                    const u64 r2s = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
                    float s0, s1v;
                    f2_unpack(r2s, s0, s1v);
                    const u64 e1 = f2_pack(ex2_sfu(-s0), ex2_sfu(-s1v));
                    const u64 e2 = f2_ex2(f2_mul(r2s, nk2));
                    a1[r] = f2_fma(e1, gj, a1[r]);
                    a2[r] = f2_fma(e2, gj, a2[r]);
                }
            }
            };
            if (per > 0.f)
                sweep(PerTag<true>{});
            else
                sweep(PerTag<false>{});
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
        float s1f = A1 * (p0 + p1), s2f = A2 * (q0 + q1);
        if (local) {  // n_i from the same rounded centred coordinates the loop used
            float mx, my, mz, unused;
            f2_unpack(xi[r], mx, unused);
            f2_unpack(yi[r], my, unused);
            f2_unpack(zi[r], mz, unused);
            const float ni = 0.25f * (mx * mx + my * my + mz * mz);  // in units of s2 when M > 0
            s1f *= exp2f(M > 0 ? -(float)M * ni : -ni);
            s2f *= exp2f(M > 0 ? -ni : -k2 * ni);
        }
        float v = warp_sum(s1f - s2f);
        if (lane == 0) partial[((int64_t)split * B + b) * n_pad + __ldg(rowperm + slot0 + r)] = v;
    }
}

// ----------------------------------------------------------------------------
// Symmetric single-trajectory kernel.  w(x_i, x_j) = w(x_j, x_i), so every unordered pair
// is evaluated once and feeds both sums: I_i += w_ij g_j and I_j += w_ij g_i.  Nodes are
// taken in Morton order (rowperm) and cut into blocks of BLK = MS_BLK (1,024) nodes, or 512
// where the operator's autotuner measured the smaller blocks faster (mid-size node sets,
// whose 1,024-node block pairs give too few CTAs); one CTA takes a block
// pair (I <= J): it gathers block J's coordinates and g into shared memory, its warps
// sweep block I's rows R at a time (the packed forms above: expanded about the warp's
// centre when its rows are close, coordinate differences otherwise), accumulate the row
// sums in registers and the column sums per warp in shared memory.  Row sums of pair
// (I, J) go to partial slot J, column sums to slot I; a diagonal pair (I = I) sweeps all
// ordered pairs of the block and writes rows only.  Every (slot, node) entry is written
// exactly once, and the stage kernel adds the n_pad / BLK slots in a fixed order, so
// results are deterministic.  Per unordered pair (expanded form, M >= 2) this costs one
// exponential and 8 FMA-pipe lane operations for two ordered pairs.
constexpr int MS_BLK = 1024;
constexpr int MS_THREADS = 256;
constexpr int MS_WARPS = MS_THREADS / 32;
// shared memory (4-byte words): column block x, y, z, g, node (5 BLK); row block node and
// precomputed row operands mx, my, mz, h1, h2, f1, f2 (8 BLK); per-pass centre and form
// (BLK: up to BLK / 4 passes x 4); per-warp column sums (MS_WARPS BLK)
constexpr size_t ms_smem_bytes(int blk) { return sizeof(float) * ((5 + 8 + 1 + MS_WARPS) * (size_t)blk); }

// Block pair of CTA t over nb blocks, enumerated as (0,0), (0,1), (1,1), (0,2), ...
__device__ __forceinline__ void sym_pair(int64_t t, int &I, int &J) {
    int64_t j = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (j * (j + 1) / 2 > t) --j;
    while ((j + 1) * (j + 2) / 2 <= t) ++j;
    J = (int)j;
    I = (int)(t - j * (j + 1) / 2);
}

// Sum R per-lane values over the warp.  Transposed butterfly: at each of the first log2(R)
// steps a lane keeps half of its rows and adds its partner's copy of them (R - 1 shuffles
// in total), then plain xor steps finish.  Every lane returns the total of row `row`.
template <int R>
__device__ __forceinline__ float warp_reduce_rows(float (&v)[R], int lane, int &row) {
    int base = 0;
    int cnt = R;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        if (cnt > 1) {
            const int h = cnt >> 1;
            const bool upper = (lane & off) != 0;
#pragma unroll
            for (int k = 0; k < R / 2; ++k) {
                if (k < h) {
                    const float send = upper ? v[k] : v[k + h];
                    const float keep = upper ? v[k + h] : v[k];
                    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                }
            }
            if (upper) base += h;
            cnt = h;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
        }
    }
    row = base;
    return v[0];
}

// D2: every node has the same z (flat domains), so the z terms of the distance vanish
// identically and are left out (bit-identical sums, one FMA fewer per pair).
template <int R, int M, int BLK, bool D2 = false>
__global__ void __launch_bounds__(MS_THREADS, 2)
mf_sym_kernel(const float *__restrict__ xyz, const float *__restrict__ g_all, const int *__restrict__ rowperm,
              int64_t n_pad, int B, int b_base, float k2, float A1, float A2, float per,
              float *__restrict__ partial, const int *__restrict__ pairs) {
    static_assert(M >= 0 && M <= 4, "form M: 0 general, 1 one Gaussian (A2 = 0), 2-4 width ratio");
    static_assert(R == 4 || R == 8, "rows per warp");
    static_assert(BLK == 512 || BLK == 1024, "block size");
    constexpr int NPASS = BLK / R;
    // Integer width ratios combine the two Gaussians per pair: with the row factors f1, f2,
    //   w_ij = A1 f1 e1 - A2 f2 e2 = (-A2 f2) (e2 + c_i e1),  c_i = -(A1 f1) / (A2 f2),
    // so one FMA forms the pair weight u = e2 + c_i e1 and one FMA each adds u g_j to the
    // row sum and u (-A2 f2 g_i) to the column sum: 8 FMA-pipe lane operations per
    // unordered pair instead of 9 (separate e1 and e2 row sums, two column FMAs).  The
    // host takes this form only while |A1 / A2| stays far from FP32 overflow (f1 <= f2
    // for M >= 2, so |c_i| <= |A1 / A2|); other kernels take the general form M = 0.
    constexpr bool CW = M >= 2;
    extern __shared__ __align__(16) float ms_smem[];
    float *xs = ms_smem, *ys = xs + BLK, *zs = ys + BLK, *gs = zs + BLK;
    int *cnode = reinterpret_cast<int *>(gs + BLK);
    int *rnode = cnode + BLK;
    float *rmx = reinterpret_cast<float *>(rnode + BLK), *rmy = rmx + BLK, *rmz = rmy + BLK;
    float *rh1 = rmz + BLK, *rh2 = rh1 + BLK, *rf1 = rh2 + BLK, *rf2 = rf1 + BLK;
    float4 *pc = reinterpret_cast<float4 *>(rf2 + BLK);  // per pass: centre, form (w = 1: expanded)
    float *colacc = reinterpret_cast<float *>(pc + BLK / 4);  // [MS_WARPS][BLK]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int I, J;
    sym_pair(pairs ? (int64_t)__ldg(pairs + blockIdx.x) : (int64_t)blockIdx.x, I, J);  // pairs: live list
    const bool diag = I == J;
    const int b = b_base + blockIdx.z;
    const float *g = g_all + (int64_t)b * n_pad;
    const float *X = xyz, *Y = xyz + n_pad, *Z = xyz + 2 * n_pad;
    const int64_t cbase = (int64_t)J * BLK, rbase = (int64_t)I * BLK;
    // exponent units: s1 (coordinates as stored), or s2 when M > 0 (times sk = s1 / s2,
    // applied once here, so r^2 and s_ij arrive as the exponent of e2)
    const float sk = M >= 2 ? sqrtf(k2) : 1.f;  // M = 1: one Gaussian, units of s1
    // gather the column block, and the row block's raw data (x, y, z, g in mx, my, mz, h1)
    for (int k = tid; k < BLK; k += MS_THREADS) {
        const int node = __ldg(rowperm + cbase + k);
        cnode[k] = node;
        xs[k] = X[node] * sk;
        ys[k] = Y[node] * sk;
        zs[k] = Z[node] * sk;
        gs[k] = g[node];
        const int rn = diag ? node : __ldg(rowperm + rbase + k);
        rnode[k] = rn;
        rmx[k] = X[rn] * sk;
        rmy[k] = Y[rn] * sk;
        rmz[k] = Z[rn] * sk;
        rh1[k] = g[rn];
    }
    for (int k = tid; k < MS_WARPS * BLK; k += MS_THREADS) colacc[k] = 0.f;
    __syncthreads();
    // period in the units of the gathered coordinates (times sk)
    const float pers = per * sk, ipers = per > 0.f ? 1.f / pers : 0.f;
    // exponent of the wider Gaussian per unit of r^2 in these units
    const float wide = M > 0 ? 1.f : fminf(1.f, k2);
    // one thread per pass: centre of the pass's R rows, the form, and the row operands.
    // Forms: 1 expanded about c (rows -2 (x_i - c)); 0 differences (rows x_i); periodic
    // kernels: 2 differences of centred coordinates (rows x_i - c), and in forms 1 and 2 the
    // columns taken at their nearest image of c.  That image is the pair's nearest image
    // unless the column lies within e (the rows' distance from c) of c's antipodal lines;
    // such a pair is at least L/2 - e apart in both images, and when the wider Gaussian's
    // exponent there exceeds 160 (log2 units) both images give exactly 0 (ex2 flushes
    // below 2^-126).  Otherwise form 3: centred differences reduced to their nearest image
    // pair by pair.  f1, f2 are the row factors 2^(-n_i) of e1 and e2 (1 outside form 1);
    // h1 = A1 f1 g_i and h2 = -A2 f2 g_i weight the row's terms in the column sums.
    for (int ps = tid; ps < NPASS; ps += MS_THREADS) {
        const int r0 = ps * R;
        float lox = 3.4e38f, loy = 3.4e38f, loz = 3.4e38f, hix = -3.4e38f, hiy = -3.4e38f, hiz = -3.4e38f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            lox = fminf(lox, rmx[r0 + r]), hix = fmaxf(hix, rmx[r0 + r]);
            loy = fminf(loy, rmy[r0 + r]), hiy = fmaxf(hiy, rmy[r0 + r]);
            loz = fminf(loz, rmz[r0 + r]), hiz = fmaxf(hiz, rmz[r0 + r]);
        }
        const float cx = 0.5f * (lox + hix), cy = 0.5f * (loy + hiy), cz = 0.5f * (loz + hiz);
        float spread = 0.f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float dx = rmx[r0 + r] - cx, dy = rmy[r0 + r] - cy, dz = rmz[r0 + r] - cz;
            spread = fmaxf(spread, dx * dx + dy * dy + dz * dz);
        }
        bool local = spread <= kSymLocalSpread * sk * sk;  // the threshold in units of s1
        int form = local ? 1 : 0;
        if (per > 0.f) {
            const float m = 0.5f * pers - sqrtf(spread);
            if (m > 0.f && wide * m * m >= 160.f) {
                form = local ? 1 : 2;
            } else {
                form = 3;
                local = false;
            }
        }
        pc[ps] = make_float4(cx, cy, cz, (float)form);
        const bool centred = form >= 2;
        const float lsc = -2.f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = r0 + r;
            const float x = local ? lsc * (rmx[k] - cx) : (centred ? rmx[k] - cx : rmx[k]);
            const float y = local ? lsc * (rmy[k] - cy) : (centred ? rmy[k] - cy : rmy[k]);
            const float z = local ? lsc * (rmz[k] - cz) : rmz[k];  // z never wraps
            const float ni = 0.25f * (x * x + y * y + z * z);  // n_i, in units of s2 when M > 0
            const float f1 = local ? exp2f(M > 0 ? -(float)M * ni : -ni) : 1.f;
            const float f2 = local ? exp2f(M > 0 ? -ni : -k2 * ni) : 1.f;
            const float gi = rh1[k];
            rmx[k] = x;
            rmy[k] = y;
            rmz[k] = z;
            // CW: h1 holds the ratio c_i of the two terms (the combined pair weight below)
            rh1[k] = CW ? -(A1 * f1) / (A2 * f2) : A1 * f1 * gi;
            rh2[k] = -A2 * f2 * gi;
            rf1[k] = A1 * f1;
            rf2[k] = -A2 * f2;
        }
    }
    __syncthreads();
    const u64 nk2 = f2_pack(-k2, -k2);
    const u64 ipp = f2_pack(ipers, ipers), npp = f2_pack(-pers, -pers), mgp = f2_pack(kRintMagic, kRintMagic);
    const float4 *xs4 = reinterpret_cast<const float4 *>(xs), *ys4 = reinterpret_cast<const float4 *>(ys);
    const float4 *zs4 = reinterpret_cast<const float4 *>(zs), *gs4 = reinterpret_cast<const float4 *>(gs);
    float4 *cw4 = reinterpret_cast<float4 *>(colacc + warp * BLK);
    float *out_rows = partial + ((int64_t)J * B + b) * n_pad;
    auto lo2 = [](float4 v) { return f2_pack(v.x, v.y); };
    auto hi2 = [](float4 v) { return f2_pack(v.z, v.w); };
    // e1, e2 of two pairs from the exponent argument (expanded s_ij or r^2)
    // e1 = e2^M by squaring on the FMA pipe.  Taking it from the SFU instead (ex2 of -M s:
    // one multiply and two more exponentials in place of two multiplies) measured slower,
    // 1.772-1.776 against 1.720 ms per sum on the 100,000-node torus (before the combined
    // pair weight), for half or all of the column pairs: the SFU results' register moves
    // cost more than the multiply saved.
    auto exps = [&](u64 arg, u64 &e1, u64 &e2) {
        float s0, s1v;
        f2_unpack(arg, s0, s1v);
        if constexpr (M == 1) {
            e1 = f2_pack(ex2_sfu(-s0), ex2_sfu(-s1v));
            e2 = 0ull;
        } else if constexpr (M > 0) {
            e2 = f2_pack(ex2_sfu(-s0), ex2_sfu(-s1v));
            const u64 sq = f2_mul(e2, e2);
            e1 = M == 2 ? sq : (M == 3 ? f2_mul(sq, e2) : f2_mul(sq, sq));
        } else {
            e1 = f2_pack(ex2_sfu(-s0), ex2_sfu(-s1v));
            e2 = f2_ex2(f2_mul(arg, nk2));
        }
    };

    for (int ps = warp; ps < NPASS; ps += MS_WARPS) {
        const int r0 = ps * R;
        const float4 c = pc[ps];
        const int form = (int)c.w;  // warp-uniform
        u64 xi[R], yi[R], zi[R], h1[R], h2[R], a1[R], a2[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            xi[r] = f2_pack(rmx[r0 + r], rmx[r0 + r]);
            yi[r] = f2_pack(rmy[r0 + r], rmy[r0 + r]);
            zi[r] = f2_pack(rmz[r0 + r], rmz[r0 + r]);
            h1[r] = f2_pack(rh1[r0 + r], rh1[r0 + r]);
            h2[r] = f2_pack(rh2[r0 + r], rh2[r0 + r]);
            a1[r] = 0ull;
            a2[r] = 0ull;
        }
        // one pair's contribution to row r's sums and to the column sum cacc
        auto accum = [&](int r, u64 e1, u64 e2, u64 gj, u64 &cacc) {
            if constexpr (M == 1) {
                a1[r] = f2_fma(e1, gj, a1[r]);
                cacc = f2_fma(e1, h1[r], cacc);
            } else if constexpr (CW) {
                const u64 u = f2_fma(e1, h1[r], e2);
                a1[r] = f2_fma(u, gj, a1[r]);
                cacc = f2_fma(u, h2[r], cacc);
            } else {
                a1[r] = f2_fma(e1, gj, a1[r]);
                a2[r] = f2_fma(e2, gj, a2[r]);
                cacc = f2_fma(e1, h1[r], f2_fma(e2, h2[r], cacc));
            }
        };
        const u64 cxp = f2_pack(c.x, c.x), cyp = f2_pack(c.y, c.y), czp = f2_pack(c.z, c.z);
        auto add_cols = [&](int q, const u64 (&cacc)[2]) {
            if (!diag) {
                float4 cv = cw4[q];
                u64 c0 = f2_add(lo2(cv), cacc[0]), c1 = f2_add(hi2(cv), cacc[1]);
                f2_unpack(c0, cv.x, cv.y);
                f2_unpack(c1, cv.z, cv.w);
                cw4[q] = cv;
            }
        };
        // form 1: expanded about c; P: columns at their nearest image of c
        auto sweep_local = [&](auto tag, auto lim) {
            constexpr bool P = decltype(tag)::value;
#pragma unroll 1
            for (int q = lane; q < (int)lim; q += 32) {
                const float4 x4 = xs4[q], y4 = ys4[q], g4 = gs4[q];
                const float4 z4 = D2 ? make_float4(0.f, 0.f, 0.f, 0.f) : zs4[q];
                u64 xt[2] = {f2_sub(lo2(x4), cxp), f2_sub(hi2(x4), cxp)};
                u64 yt[2] = {f2_sub(lo2(y4), cyp), f2_sub(hi2(y4), cyp)};
                const u64 zt[2] = {f2_sub(lo2(z4), czp), f2_sub(hi2(z4), czp)};
                if constexpr (P) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        xt[h] = f2_wrap(xt[h], ipp, npp, mgp);
                        yt[h] = f2_wrap(yt[h], ipp, npp, mgp);
                    }
                }
                const u64 gj[2] = {lo2(g4), hi2(g4)};
                u64 nj[2], cacc[2] = {0ull, 0ull};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    nj[h] = f2_fma(yt[h], yt[h], f2_mul(xt[h], xt[h]));
                    if constexpr (!D2) nj[h] = f2_fma(zt[h], zt[h], nj[h]);
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const u64 zz = D2 ? nj[h] : f2_fma(zi[r], zt[h], nj[h]);
                        const u64 sij = f2_fma(xi[r], xt[h], f2_fma(yi[r], yt[h], zz));
                        u64 e1, e2;
                        exps(sij, e1, e2);
                        accum(r, e1, e2, gj[h], cacc[h]);
                    }
                }
                add_cols(q, cacc);
            }
        };
        // forms 0, 2, 3: coordinate differences; CEN: rows centred on c and columns' x, y at
        // their nearest image of c (forms 2, 3); PW: each pair's x, y differences reduced to
        // their nearest image (form 3)
        auto sweep_diff = [&](auto tag_c, auto tag_w, auto lim) {
            constexpr bool CEN = decltype(tag_c)::value, PW = decltype(tag_w)::value;
#pragma unroll 1
            for (int q = lane; q < (int)lim; q += 32) {
                const float4 x4 = xs4[q], y4 = ys4[q], g4 = gs4[q];
                const float4 z4 = D2 ? make_float4(0.f, 0.f, 0.f, 0.f) : zs4[q];
                u64 xj[2] = {lo2(x4), hi2(x4)}, yj[2] = {lo2(y4), hi2(y4)};
                const u64 zj[2] = {lo2(z4), hi2(z4)};
                if constexpr (CEN) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        xj[h] = f2_wrap(f2_sub(xj[h], cxp), ipp, npp, mgp);
                        yj[h] = f2_wrap(f2_sub(yj[h], cyp), ipp, npp, mgp);
                    }
                }
                const u64 gj[2] = {lo2(g4), hi2(g4)};
                u64 cacc[2] = {0ull, 0ull};
#pragma unroll
                for (int r = 0; r < R; ++r) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        u64 dx = f2_sub(xi[r], xj[h]), dy = f2_sub(yi[r], yj[h]);
                        const u64 dz = f2_sub(zi[r], zj[h]);
                        if constexpr (PW) {
                            dx = f2_wrap(dx, ipp, npp, mgp);
                            dy = f2_wrap(dy, ipp, npp, mgp);
                        }
                        const u64 r2xy = f2_fma(dy, dy, f2_mul(dx, dx));
                        const u64 r2s = D2 ? r2xy : f2_fma(dz, dz, r2xy);
                        u64 e1, e2;
                        exps(r2s, e1, e2);
                        accum(r, e1, e2, gj[h], cacc[h]);
                    }
                }
                add_cols(q, cacc);
            }
        };
        // each lane takes 4 consecutive columns (two f32x2 pairs) per step.  Every block is
        // swept in full, padding included (g = 0 there): a second, trimmed copy of the loops
        // for the last block measured 2.5 % slower on the 100,000-node torus (1.763 against
        // 1.720 ms per sum, before the combined pair weight), more than its 0.7 % of padded
        // pairs
        auto run = [&](auto lim) {
            if (form == 1) {
                if (per > 0.f)
                    sweep_local(PerTag<true>{}, lim);
                else
                    sweep_local(PerTag<false>{}, lim);
            } else if (form == 0) {
                sweep_diff(PerTag<false>{}, PerTag<false>{}, lim);
            } else if (form == 2) {
                sweep_diff(PerTag<true>{}, PerTag<false>{}, lim);
            } else {
                sweep_diff(PerTag<true>{}, PerTag<true>{}, lim);
            }
        };
        run(CInt<BLK / 4>{});
        float v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float p0, p1, q0, q1;
            f2_unpack(a1[r], p0, p1);
            if constexpr (CW) {
                v[r] = rf2[r0 + r] * (p0 + p1);
            } else {
                f2_unpack(a2[r], q0, q1);
                v[r] = rf1[r0 + r] * (p0 + p1) + rf2[r0 + r] * (q0 + q1);
            }
        }
        int row;
        const float tot = warp_reduce_rows<R>(v, lane, row);
        if ((lane & (32 / R - 1)) == 0) out_rows[rnode[r0 + row]] = tot;
    }
    if (diag) return;
    __syncthreads();
    float *out_cols = partial + ((int64_t)I * B + b) * n_pad;
    for (int k = tid; k < BLK; k += MS_THREADS) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < MS_WARPS; ++w) v += colacc[w * BLK + k];
        out_cols[cnode[k]] = v;
    }
}

// ----------------------------------------------------------------------------
// Symmetric adjoint pair kernel (one trajectory b).  W is symmetric, so each unordered
// pair of nodes is evaluated once, as in the forward symmetric kernel: one CTA per pair of
// 1024-node Morton blocks (I <= J), rows of block I swept R at a time against block J in
// shared memory, expanded about the pass's centre when its rows are close.  Per pair it
//   * adds e1, e2 times nu to the row sums (W nu)_i and, per warp in shared memory, to the
//     column sums (W nu)_j: row sums go to slot J, column sums to slot I of wpart, the
//     stage epilogue adds the slots in a fixed order;
//   * adds the pair's share of the kernel-parameter sums
//         P1 = sum nu_i g_j e1, Q1 = sum nu_i g_j r^2 e1, P2 = sum nu_i g_j e2, Q2 = ... r^2 e2
//     over ordered pairs: off the diagonal an unordered pair carries the weight
//     nu_i g_j + nu_j g_i, on a diagonal block pair every ordered pair is swept with
//     nu_i g_j.  The row's factor nu_i (or g_i) comes out of its sum over j, so per pair
//     the lane only accumulates sum e g_j, sum arg e g_j and sum arg e nu_j per row
//     (sum e nu_j is the W nu row sum), with arg = r^2 - n_i; the pass end forms the
//     four sums from them.  Each CTA writes its four sums (r^2 in exponent units: of s2
//     when M > 0, else of s1) to gpart; a fixed-order FP64 reduction adds them.
constexpr size_t as_smem_floats(int blk) { return (size_t)(5 + 14 + 1 + MS_WARPS) * blk; }

// R = 4: two CTAs per SM (128 registers); R = 8: one CTA per SM with the whole register
// file (eight rows' accumulators, more independent work per warp, fewer warps).  BLK: node
// block of 1,024 or 512 (four times the CTAs, for node sets whose 1,024-node block pairs
// leave the last wave of CTAs partly empty).
template <int R, int M, int BLK>
__global__ void __launch_bounds__(MS_THREADS, R >= 8 ? 1 : 2)
adj_sym_kernel(const float *__restrict__ xyz, const float2 *__restrict__ vg_all, const int *__restrict__ rowperm,
               int64_t n_pad, int B, int b, float k2, float A1, float A2, float per,
               float *__restrict__ wpart, float *__restrict__ gpart, const int *__restrict__ pairs) {
    static_assert(M == 0 || (M >= 2 && M <= 4), "width ratio M must be 0 (general), 2, 3 or 4");
    static_assert(R == 4 || R == 8, "rows per warp");
    static_assert(BLK == 512 || BLK == 1024, "block size");
    constexpr int NPASS = BLK / R;
    // CW (integer width ratios, A2 != 0): per pair the W nu sums take the combined weight
    // u = e2 + c_i e1 (c_i = -A1 f1 / (A2 f2), as in mf_sym_kernel), and the parameter sums
    // the symmetric pair weight p_ij = nu_i g_j + g_i nu_j, formed once per pair: per row
    // the lane keeps U = sum u nu_j (the W nu row sum), sum e1 p, sum e2 p, sum arg e1 p and
    // sum arg e2 p -- 16 FMA-pipe instructions per row and column pair instead of 17, and
    // five accumulators per row instead of eight.  The host takes this form only while
    // |A1 / A2| <= 2^100; otherwise, and for A2 = 0, the general form M = 0.
    constexpr bool CW = M >= 2;
    extern __shared__ __align__(16) float as_smem[];
    // column block: x, y, z, nu, g (floats), node (int)
    float *xs = as_smem, *ys = xs + BLK, *zs = ys + BLK, *vs = zs + BLK, *gsm = vs + BLK;
    int *cnode = reinterpret_cast<int *>(gsm + BLK);
    // row block: node; per row (mx, my, mz, n_i), (h1, h1, h2, h2) -- the column-sum weights
    // A1 f1 nu_i and -A2 f2 nu_i -- and (v1, u1, v2, u2), as float4
    int *rnode = cnode + BLK;
    float4 *rgeo = reinterpret_cast<float4 *>(rnode + BLK);
    float4 *rwn = rgeo + BLK, *rgw = rwn + BLK;
    float4 *pc = rgw + BLK;                               // per pass: centre, form
    float *colacc = reinterpret_cast<float *>(pc + BLK / 4);  // [MS_WARPS][BLK]
    __shared__ float gred[MS_WARPS][4];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int I, J;
    sym_pair(pairs ? (int64_t)__ldg(pairs + blockIdx.x) : (int64_t)blockIdx.x, I, J);  // pairs: live list
    const bool diag = I == J;
    const float2 *vg = vg_all + (int64_t)b * n_pad;
    const float *X = xyz, *Y = xyz + n_pad, *Z = xyz + 2 * n_pad;
    const int64_t cbase = (int64_t)J * BLK, rbase = (int64_t)I * BLK;
    // exponent units: s1, or s2 when M > 0 (coordinates times sk = s1 / s2, once here)
    const float sk = M > 0 ? sqrtf(k2) : 1.f;
    for (int k = tid; k < BLK; k += MS_THREADS) {
        const int node = __ldg(rowperm + cbase + k);
        cnode[k] = node;
        xs[k] = X[node] * sk;
        ys[k] = Y[node] * sk;
        zs[k] = Z[node] * sk;
        const float2 p = vg[node];
        vs[k] = p.x;
        gsm[k] = p.y;
        const int rn = diag ? node : __ldg(rowperm + rbase + k);
        rnode[k] = rn;
        const float2 pr = diag ? p : vg[rn];
        rgeo[k] = make_float4(X[rn] * sk, Y[rn] * sk, Z[rn] * sk, 0.f);
        rgw[k] = make_float4(pr.x, pr.y, 0.f, 0.f);
    }
    for (int k = tid; k < MS_WARPS * BLK; k += MS_THREADS) colacc[k] = 0.f;
    __syncthreads();
    // one thread per pass: centre, form and the rows' operands (see mf_sym_kernel)
    for (int ps = tid; ps < NPASS; ps += MS_THREADS) {
        const int r0 = ps * R;
        float lox = 3.4e38f, loy = 3.4e38f, loz = 3.4e38f, hix = -3.4e38f, hiy = -3.4e38f, hiz = -3.4e38f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float4 p = rgeo[r0 + r];
            lox = fminf(lox, p.x), hix = fmaxf(hix, p.x);
            loy = fminf(loy, p.y), hiy = fmaxf(hiy, p.y);
            loz = fminf(loz, p.z), hiz = fmaxf(hiz, p.z);
        }
        const float cx = 0.5f * (lox + hix), cy = 0.5f * (loy + hiy), cz = 0.5f * (loz + hiz);
        float spread = 0.f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float4 p = rgeo[r0 + r];
            const float dx = p.x - cx, dy = p.y - cy, dz = p.z - cz;
            spread = fmaxf(spread, dx * dx + dy * dy + dz * dz);
        }
        // the threshold in units of s1; periodic distances take the difference form
        const bool local = spread <= kSymLocalSpread * sk * sk && !(per > 0.f);
        pc[ps] = make_float4(cx, cy, cz, local ? 1.f : 0.f);
        const float lsc = -2.f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = r0 + r;
            const float4 p = rgeo[k];
            const float x = local ? lsc * (p.x - cx) : p.x;
            const float y = local ? lsc * (p.y - cy) : p.y;
            const float z = local ? lsc * (p.z - cz) : p.z;
            const float ni = local ? 0.25f * (x * x + y * y + z * z) : 0.f;  // exponent units
            const float f1 = local ? exp2f(M > 0 ? -(float)M * ni : -ni) : 1.f;
            const float f2 = local ? exp2f(M > 0 ? -ni : -k2 * ni) : 1.f;
            const float nu = rgw[k].x, gi = rgw[k].y;
            rgeo[k] = make_float4(x, y, z, ni);
            const float h1 = A1 * f1 * nu, h2 = -A2 * f2 * nu;
            if constexpr (CW) {  // (c_i, -, h2): ratio and column weight; (nu_i, g_i): pair weight
                rwn[k] = make_float4(-(A1 * f1) / (A2 * f2), 0.f, h2, h2);
                rgw[k] = make_float4(nu, diag ? 0.f : gi, 0.f, 0.f);
            } else {
                rwn[k] = make_float4(h1, h1, h2, h2);
                rgw[k] = make_float4(f1 * nu, diag ? 0.f : f1 * gi, f2 * nu, diag ? 0.f : f2 * gi);
            }
        }
    }
    __syncthreads();
    const u64 nk2 = f2_pack(-k2, -k2);
    const float pers = per * sk, ipers = per > 0.f ? 1.f / pers : 0.f;
    const u64 ipp = f2_pack(ipers, ipers), npp = f2_pack(-pers, -pers), mgp = f2_pack(kRintMagic, kRintMagic);
    const u64 *xs2 = reinterpret_cast<const u64 *>(xs), *ys2 = reinterpret_cast<const u64 *>(ys);
    const u64 *zs2 = reinterpret_cast<const u64 *>(zs), *vs2 = reinterpret_cast<const u64 *>(vs);
    const u64 *gs2 = reinterpret_cast<const u64 *>(gsm);
    u64 *cw2 = reinterpret_cast<u64 *>(colacc + warp * BLK);
    float *out_rows = wpart + ((int64_t)J * B + b) * n_pad;
    auto exps = [&](u64 arg, u64 &e1, u64 &e2) {
        float s0, s1v;
        f2_unpack(arg, s0, s1v);
        if constexpr (M > 0) {
            e2 = f2_pack(ex2_sfu(-s0), ex2_sfu(-s1v));
            const u64 sq = f2_mul(e2, e2);
            e1 = M == 2 ? sq : (M == 3 ? f2_mul(sq, e2) : f2_mul(sq, sq));
        } else {
            e1 = f2_pack(ex2_sfu(-s0), ex2_sfu(-s1v));
            e2 = f2_ex2(f2_mul(arg, nk2));
        }
    };
    float P1 = 0.f, Q1 = 0.f, P2 = 0.f, Q2 = 0.f;  // per lane, over all its pairs
    for (int ps = warp; ps < NPASS; ps += MS_WARPS) {
        const int r0 = ps * R;
        const float4 c = pc[ps];
        const bool local = c.w != 0.f;
        // per row, over the lane's columns j (e1, e2 without the row factors):
        //   a = sum e nu_j, b = sum e g_j, c = sum arg e g_j, d = sum arg e nu_j
        // CW: a1 = U, b1, b2 = sum e p, c1, c2 = sum arg e p; pn, pg = nu_i, g_i; h1 = c_i
        u64 xi[R], yi[R], zi[R], h1[R], h2[R], a1[R], a2[R], b1[R], b2[R], c1[R], c2[R], d1[R], d2[R];
        u64 pn[R], pg[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float4 p = rgeo[r0 + r], w = rwn[r0 + r];
            xi[r] = f2_pack(p.x, p.x);
            yi[r] = f2_pack(p.y, p.y);
            zi[r] = f2_pack(p.z, p.z);
            h1[r] = f2_pack(w.x, w.x);
            h2[r] = f2_pack(w.z, w.z);
            if constexpr (CW) {
                const float4 q = rgw[r0 + r];
                pn[r] = f2_pack(q.x, q.x);
                pg[r] = f2_pack(q.y, q.y);
                a1[r] = b1[r] = b2[r] = c1[r] = c2[r] = 0ull;
            } else {
                a1[r] = a2[r] = b1[r] = b2[r] = c1[r] = c2[r] = d1[r] = d2[r] = 0ull;
            }
        }
        const u64 cxp = f2_pack(c.x, c.x), cyp = f2_pack(c.y, c.y), czp = f2_pack(c.z, c.z);
        // per (row, column pair): e1, e2 from the exponent argument arg (r^2 - n_i in the
        // expanded form, r^2 otherwise), then the W nu and row-sum updates
        auto pair = [&](int r, u64 arg, u64 vj, u64 gj, u64 &cacc) {
            u64 e1, e2;
            exps(arg, e1, e2);
            const u64 s1e = f2_mul(arg, e1), s2e = f2_mul(arg, e2);
            if constexpr (CW) {
                const u64 u = f2_fma(e1, h1[r], e2);
                a1[r] = f2_fma(u, vj, a1[r]);
                cacc = f2_fma(u, h2[r], cacc);
                const u64 pw = f2_fma(pn[r], gj, f2_mul(pg[r], vj));
                b1[r] = f2_fma(e1, pw, b1[r]);
                b2[r] = f2_fma(e2, pw, b2[r]);
                c1[r] = f2_fma(s1e, pw, c1[r]);
                c2[r] = f2_fma(s2e, pw, c2[r]);
            } else {
                a1[r] = f2_fma(e1, vj, a1[r]);
                a2[r] = f2_fma(e2, vj, a2[r]);
                cacc = f2_fma(e1, h1[r], f2_fma(e2, h2[r], cacc));
                b1[r] = f2_fma(e1, gj, b1[r]);
                b2[r] = f2_fma(e2, gj, b2[r]);
                c1[r] = f2_fma(s1e, gj, c1[r]);
                d1[r] = f2_fma(s1e, vj, d1[r]);
                c2[r] = f2_fma(s2e, gj, c2[r]);
                d2[r] = f2_fma(s2e, vj, d2[r]);
            }
        };
        auto sweep_local = [&](auto lim) {
#pragma unroll 1
            for (int jp = lane; jp < (int)lim; jp += 32) {
                const u64 xt = f2_sub(xs2[jp], cxp), yt = f2_sub(ys2[jp], cyp), zt = f2_sub(zs2[jp], czp);
                const u64 nj = f2_fma(zt, zt, f2_fma(yt, yt, f2_mul(xt, xt)));
                const u64 vj = vs2[jp], gj = gs2[jp];
                u64 cacc = 0ull;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    pair(r, f2_fma(xi[r], xt, f2_fma(yi[r], yt, f2_fma(zi[r], zt, nj))), vj, gj, cacc);
                if (!diag) cw2[jp] = f2_add(cw2[jp], cacc);
            }
        };
        // every block is swept in full, padding included (nu = g = 0 there): stopping at the
        // last real column measured no faster (809 against 811 ms for the 200-step gradient
        // at n = 40,000, whose padding is 5 % of the pairs)
        if (local) {
            sweep_local(CInt<BLK / 2>{});
        } else {
            auto sweep = [&](auto tag, auto lim) {
                constexpr bool P = decltype(tag)::value;
#pragma unroll 1
            for (int jp = lane; jp < (int)lim; jp += 32) {
                const u64 xj = xs2[jp], yj = ys2[jp], zj = zs2[jp], vj = vs2[jp], gj = gs2[jp];
                u64 cacc = 0ull;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    u64 dx = f2_sub(xi[r], xj), dy = f2_sub(yi[r], yj);
                    const u64 dz = f2_sub(zi[r], zj);
                    if constexpr (P) {
                        dx = f2_wrap(dx, ipp, npp, mgp);
                        dy = f2_wrap(dy, ipp, npp, mgp);
                    }
                    pair(r, f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx))), vj, gj, cacc);
                }
                if (!diag) cw2[jp] = f2_add(cw2[jp], cacc);
            }
            };
            if (per > 0.f)
                sweep(PerTag<true>{}, CInt<BLK / 2>{});
            else
                sweep(PerTag<false>{}, CInt<BLK / 2>{});
        }
        auto fold = [](u64 x) {
            float lo, hi;
            f2_unpack(x, lo, hi);
            return lo + hi;
        };
        float v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float ni = rgeo[r0 + r].w;
            // the row factors 2^(-n_i) of e1 and e2 as in the pass set-up (n_i = 0 outside
            // the expanded form, so both are 1 there)
            const float f1 = exp2f(M > 0 ? -(float)M * ni : -ni), f2 = exp2f(M > 0 ? -ni : -k2 * ni);
            if constexpr (CW) {
                const float P1s = fold(b1[r]), P2s = fold(b2[r]);
                v[r] = (-A2 * f2) * fold(a1[r]);
                P1 += f1 * P1s;
                Q1 += f1 * (fold(c1[r]) + ni * P1s);
                P2 += f2 * P2s;
                Q2 += f2 * (fold(c2[r]) + ni * P2s);
                continue;
            }
            const float A1s = fold(a1[r]), A2s = fold(a2[r]), B1s = fold(b1[r]), B2s = fold(b2[r]);
            const float4 q = rgw[r0 + r];
            v[r] = (A1 * f1) * A1s + (-A2 * f2) * A2s;
            // pair weight e (nu_i g_j + g_i nu_j) with the row factors: q = (f1 nu_i, f1 g_i,
            // f2 nu_i, f2 g_i), g_i = 0 on diagonal block pairs; r^2 = arg + n_i
            P1 += q.x * B1s + q.y * A1s;
            Q1 += q.x * (fold(c1[r]) + ni * B1s) + q.y * (fold(d1[r]) + ni * A1s);
            P2 += q.z * B2s + q.w * A2s;
            Q2 += q.z * (fold(c2[r]) + ni * B2s) + q.w * (fold(d2[r]) + ni * A2s);
        }
        int row;
        const float tot = warp_reduce_rows<R>(v, lane, row);
        if ((lane & (32 / R - 1)) == 0) out_rows[rnode[r0 + row]] = tot;
    }
    // the CTA's parameter sums: lanes, then warps, in a fixed order
    float gs4[4] = {P1, Q1, P2, Q2};
#pragma unroll
    for (int k = 0; k < 4; ++k) gs4[k] = warp_sum(gs4[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) gred[warp][k] = gs4[k];
    __syncthreads();
    if (tid < 4) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < MS_WARPS; ++w) s += gred[w][tid];
        gpart[((int64_t)b * gridDim.x + blockIdx.x) * 4 + tid] = s;
    }
    if (diag) return;
    float *out_cols = wpart + ((int64_t)I * B + b) * n_pad;
    for (int k = tid; k < BLK; k += MS_THREADS) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < MS_WARPS; ++w) s += colacc[w * BLK + k];
        out_cols[cnode[k]] = s;
    }
}

// ----------------------------------------------------------------------------
// split planner: (row blocks x column splits) items of equal cost; pick the number
// of splits (at most max_splits) that best fills whole waves of resident blocks.
SplitPlan plan_splits(int64_t n_pad, int rows_per_block, int tile_cols, int resident_blocks_per_sm, int max_splits) {
    SplitPlan p{};
    p.rows_per_block = rows_per_block;
    p.row_blocks = n_pad / rows_per_block;
    const int64_t tiles = n_pad / tile_cols;
    const int64_t slots = (int64_t)num_sms() * std::max(1, resident_blocks_per_sm);
    double best = -1.0;
    int best_s = 1;
    const int64_t smax = std::min<int64_t>(tiles, std::max(1, max_splits));
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
template <int R, int M, int BLK = 1024, bool D2 = false>
static cudaError_t set_sym_attr() {
    return cudaFuncSetAttribute(mf_sym_kernel<R, M, BLK, D2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ms_smem_bytes(BLK));
}

template <int R, int M, int BLK>
static cudaError_t set_adj_attr() {
    return cudaFuncSetAttribute(adj_sym_kernel<R, M, BLK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(as_smem_floats(BLK) * sizeof(float)));
}

// The attributes belong to the device's context: set once per device (under a lock, so that
// concurrent first calls on one device do not race), with that device current.
static nf_status mf_init_attrs_device();

nf_status mf_init_attrs() {
    static std::mutex mu;
    static bool done[64] = {false};
    const int d = device_id();
    if (d < 0 || d >= 64) return mf_init_attrs_device();
    std::lock_guard<std::mutex> lock(mu);
    if (done[d]) return NF_OK;
    NF_TRY(mf_init_attrs_device());
    done[d] = true;
    return NF_OK;
}

static nf_status mf_init_attrs_device() {
    NF_TRY(dense_init_attrs());
    NF_CUDA_TRY((set_adj_attr<4, 0, 1024>()));
    NF_CUDA_TRY((set_adj_attr<4, 2, 1024>()));
    NF_CUDA_TRY((set_adj_attr<4, 3, 1024>()));
    NF_CUDA_TRY((set_adj_attr<4, 4, 1024>()));
    NF_CUDA_TRY((set_adj_attr<8, 0, 1024>()));
    NF_CUDA_TRY((set_adj_attr<8, 2, 1024>()));
    NF_CUDA_TRY((set_adj_attr<8, 3, 1024>()));
    NF_CUDA_TRY((set_adj_attr<8, 4, 1024>()));
    NF_CUDA_TRY((set_adj_attr<4, 0, 512>()));
    NF_CUDA_TRY((set_adj_attr<4, 2, 512>()));
    NF_CUDA_TRY((set_adj_attr<4, 3, 512>()));
    NF_CUDA_TRY((set_adj_attr<4, 4, 512>()));
    NF_CUDA_TRY((set_adj_attr<8, 0, 512>()));
    NF_CUDA_TRY((set_adj_attr<8, 2, 512>()));
    NF_CUDA_TRY((set_adj_attr<8, 3, 512>()));
    NF_CUDA_TRY((set_adj_attr<8, 4, 512>()));
    NF_CUDA_TRY((set_sym_attr<4, 0>()));
    NF_CUDA_TRY((set_sym_attr<4, 1>()));
    NF_CUDA_TRY((set_sym_attr<8, 1>()));
    NF_CUDA_TRY((set_sym_attr<4, 2>()));
    NF_CUDA_TRY((set_sym_attr<4, 3>()));
    NF_CUDA_TRY((set_sym_attr<4, 4>()));
    NF_CUDA_TRY((set_sym_attr<8, 0>()));
    NF_CUDA_TRY((set_sym_attr<8, 2>()));
    NF_CUDA_TRY((set_sym_attr<8, 3>()));
    NF_CUDA_TRY((set_sym_attr<8, 4>()));
    NF_CUDA_TRY((set_sym_attr<8, 0, 512>()));
    NF_CUDA_TRY((set_sym_attr<8, 1, 512>()));
    NF_CUDA_TRY((set_sym_attr<8, 2, 512>()));
    NF_CUDA_TRY((set_sym_attr<8, 3, 512>()));
    NF_CUDA_TRY((set_sym_attr<8, 4, 512>()));
    NF_CUDA_TRY((set_sym_attr<8, 0, 1024, true>()));
    NF_CUDA_TRY((set_sym_attr<8, 1, 1024, true>()));
    NF_CUDA_TRY((set_sym_attr<8, 2, 1024, true>()));
    NF_CUDA_TRY((set_sym_attr<8, 3, 1024, true>()));
    NF_CUDA_TRY((set_sym_attr<8, 4, 1024, true>()));
    NF_CUDA_TRY((set_mf_attr<1, 2>()));
    NF_CUDA_TRY((set_mf_attr<2, 2>()));
    NF_CUDA_TRY((set_mf_attr<4, 2>()));
    NF_CUDA_TRY((set_mf_attr<8, 2>()));
    NF_CUDA_TRY((set_mf_attr<1, 4>()));
    NF_CUDA_TRY((set_mf_attr<2, 4>()));
    NF_CUDA_TRY((set_mf_attr<4, 4>()));
    NF_CUDA_TRY((set_mf_attr<8, 4>()));
    NF_CUDA_TRY((set_mf_attr<16, 2>()));
    NF_CUDA_TRY((set_mf_attr<16, 4>()));
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
                                                         k.A1, k.A2, k.period, op->partial, op->err);
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

// The kernel's period in the units of the pre-scaled coordinates (times sqrt(log2 e) / s1,
// as the node packing scales them); 0 for the Euclidean distance.
static float scaled_period(const nf_kernel &k) {
    return k.period > 0.f ? k.period * (std::sqrt(1.4426950408889634f) / k.s1) : 0.f;
}

// Form of the symmetric kernel: 1 for a single Gaussian (A2 = 0), else the width ratio.
// The width-ratio forms combine the two Gaussians through the ratio -A1 f1 / (A2 f2) per
// row, which stays finite while |A1 / A2| <= 2^100; beyond that the general form.
static int mf_width_ratio(const nf_kernel &k);
static int sym_form(const nf_kernel &k) {
    if (k.A2 == 0.f) return 1;
    const int m = mf_width_ratio(k);
    if (m >= 2 && !(std::fabs((double)k.A1) <= 0x1p100 * std::fabs((double)k.A2))) return 0;
    return m;
}

// Integer width ratio m = s2^2 / s1^2 in {2, 3, 4} (to FP32 rounding of the k2 the kernel
// receives), else 0: selects the one-exponential form of the packed kernel.
static int mf_width_ratio(const nf_kernel &k) {
    const float k2 = (k.s1 * k.s1) / (k.s2 * k.s2);
    for (int m = 2; m <= 4; ++m)
        if (std::fabs((double)m * (double)k2 - 1.0) <= 4.0 * (double)FLT_EPSILON) return m;
    return 0;
}

template <int R, int TJ>
static int packed_resident() {
    int nb0 = 0, nb4 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb0, mf_pair_packed_kernel<R, TJ, 0>, MF_THREADS, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb4, mf_pair_packed_kernel<R, TJ, 4>, MF_THREADS, 0);
    return std::max(std::min(nb0, nb4), 1);
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
#define NF_PACKED_ARGS \
    op->xyz, op->g, op->rowperm, op->n_pad, B, b_base, pl.jchunk, k2, k.A1, k.A2, scaled_period(k), op->partial, \
        op->err
    switch (mf_width_ratio(k)) {
        case 2: mf_pair_packed_kernel<R, TJ, 2><<<grid, MF_THREADS, 0, s>>>(NF_PACKED_ARGS); break;
        case 3: mf_pair_packed_kernel<R, TJ, 3><<<grid, MF_THREADS, 0, s>>>(NF_PACKED_ARGS); break;
        case 4: mf_pair_packed_kernel<R, TJ, 4><<<grid, MF_THREADS, 0, s>>>(NF_PACKED_ARGS); break;
        default: mf_pair_packed_kernel<R, TJ, 0><<<grid, MF_THREADS, 0, s>>>(NF_PACKED_ARGS); break;
    }
#undef NF_PACKED_ARGS
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

// Launch shape of the packed kernel (single trajectories inside a multi-trajectory call):
// small node sets want more, smaller blocks.
static int default_variant(int64_t n_pad) { return n_pad >= 16384 ? 3 : 0; }

// ---- symmetric kernel launch (B = 1)
// Block pairs and slots of the forward symmetric kernel at the operator's block size
// (1,024 nodes, or 512 where the autotuner found the smaller blocks faster: more CTAs for
// mid-size node sets).
static int64_t sym_pairs(const nf_operator *op) {
    const int64_t nb = op->n_pad / op->sym_blk;
    return nb * (nb + 1) / 2;
}
static int64_t sym_pairs_1024(const nf_operator *op) {
    const int64_t nb = op->n_pad / MS_BLK;
    return nb * (nb + 1) / 2;
}

template <int R, int BLK, bool D2 = false>
static void launch_sym_rb(nf_operator *op, int B, int b_base, cudaStream_t s) {
    const nf_kernel &k = op->kp;
    const float k2 = (k.s1 * k.s1) / (k.s2 * k.s2);
    // blockIdx.z: trajectory b_base + z of the B in the partial-sum layout
    dim3 grid((unsigned)(op->mf_cull ? op->cull_live : sym_pairs(op)), 1, (unsigned)(B - b_base));
    const size_t smem = ms_smem_bytes(BLK);
#define NF_SYM_ARGS                                                                                       \
    op->xyz, op->g, op->rowperm, op->n_pad, B, b_base, k2, k.A1, k.A2, scaled_period(k), op->partial, \
        (op->mf_cull ? op->cull_pairs : nullptr)
    switch (sym_form(k)) {
        case 1: mf_sym_kernel<R, 1, BLK, D2><<<grid, MS_THREADS, smem, s>>>(NF_SYM_ARGS); break;
        case 2: mf_sym_kernel<R, 2, BLK, D2><<<grid, MS_THREADS, smem, s>>>(NF_SYM_ARGS); break;
        case 3: mf_sym_kernel<R, 3, BLK, D2><<<grid, MS_THREADS, smem, s>>>(NF_SYM_ARGS); break;
        case 4: mf_sym_kernel<R, 4, BLK, D2><<<grid, MS_THREADS, smem, s>>>(NF_SYM_ARGS); break;
        default: mf_sym_kernel<R, 0, BLK, D2><<<grid, MS_THREADS, smem, s>>>(NF_SYM_ARGS); break;
    }
#undef NF_SYM_ARGS
}

static nf_status launch_sym(nf_operator *op, int B, int b_base, cudaStream_t s) {
    if (op->sym_blk == 512)
        launch_sym_rb<8, 512>(op, B, b_base, s);
    else if (op->mf_sym_r == 4)
        launch_sym_rb<4, 1024>(op, B, b_base, s);
    else if (op->planar)
        launch_sym_rb<8, 1024, true>(op, B, b_base, s);
    else
        launch_sym_rb<8, 1024>(op, B, b_base, s);
    NF_CUDA_TRY(cudaGetLastError());
    return NF_OK;
}

// Adjoint pair sums of trajectory b over all 1,024-node block pairs (see adj_sym_kernel):
// W nu slots into wpart [n_pad / 1024][B][n_pad], parameter sums into gpart [B][pairs][4]
// with r^2 in exponent units; *r2_phys receives the factor to physical r^2.
// The adjoint kernel's node block: the tuned one, or 1,024 when culling (its live-pair lists
// are built over 1,024-node blocks).
static int adj_block(const nf_operator *op) {
    return (op->mf_cull && op->adj_pairs) || op->adj_blk == 0 ? MS_BLK : op->adj_blk;
}
int64_t sym_pair_count(const nf_operator *op) {
    const int64_t nb = op->n_pad / adj_block(op);
    return nb * (nb + 1) / 2;
}
int adj_slots(const nf_operator *op) { return (int)(op->n_pad / adj_block(op)); }
int64_t adj_pair_capacity(const nf_operator *op) {
    const int64_t nb = op->n_pad / 512;
    return nb * (nb + 1) / 2;
}
int adj_slot_capacity(const nf_operator *op) { return (int)(op->n_pad / 512); }
int sym_slots(const nf_operator *op) { return (int)(op->n_pad / op->sym_blk); }

// Up to kSymMaxB trajectories take the symmetric kernel, one launch with a grid z per
// trajectory: each trajectory's pairs are evaluated once, which beats the multi-trajectory
// kernels (ordered pairs, exponentials shared across trajectories) until about four
// trajectories (measured at n = 1e5: B = 2 in 4.9 ms and B = 3 in 7.7 ms there, against
// 1.8 ms per symmetric trajectory; B = 4 in 5.4 ms).
constexpr int kSymMaxB = 3;

// One trajectory takes the symmetric kernel when it has at least 2/3 as many block pairs as
// the GPU has SMs; smaller node sets (below ~13,300 nodes on 152 SMs) have too few block
// pairs to fill the GPU and take the packed row-block x column-split kernel instead, which
// evaluates ordered pairs but spreads them over many more CTAs (measured crossover on GB300:
// packed 0.119 ms vs symmetric 0.130 ms at n = 12,000; 0.155 vs 0.131 ms at n = 16,384).
// The automatic schedule also keeps the symmetric partial sums (one slot of n_pad floats per
// 1,024-node block, growing as n^2) within an eighth of the device memory: beyond that (n
// above about 3 million on a GB300) the packed kernel, whose layout grows with its column
// splits only, takes over.
static bool sym_layout_fits(const nf_operator *op) {
    static std::atomic<size_t> budget[64];  // per device, an eighth of its memory
    const int d = device_id();
    size_t b = (d >= 0 && d < 64) ? budget[d].load() : 0;
    if (!b) {
        size_t freeb = 0, total = 0;
        b = (cudaMemGetInfo(&freeb, &total) == cudaSuccess && total > 0) ? total / 8 : ((size_t)8 << 30);
        if (d >= 0 && d < 64) budget[d].store(b);
    }
    return (double)(op->n_pad / MS_BLK) * (double)op->n_pad * sizeof(float) <= (double)b;
}

static bool use_sym(const nf_operator *op) {
    if (op->mf_sched == NF_MF_SYMMETRIC) return true;
    if (op->mf_sched == NF_MF_PACKED) return false;
    return 3 * sym_pairs_1024(op) >= 2 * (int64_t)num_sms() && sym_layout_fits(op);
}

// Form of the adjoint kernel: the width ratio m in {2, 3, 4} (combined W nu weight through the
// ratio -A1 f1 / (A2 f2)) while A2 != 0 and |A1 / A2| <= 2^100, else the general form 0.
static int adj_form(const nf_kernel &k) {
    const int m = mf_width_ratio(k);
    if (m >= 2 && (k.A2 == 0.f || !(std::fabs((double)k.A1) <= 0x1p100 * std::fabs((double)k.A2)))) return 0;
    return m;
}

nf_status launch_adj_sym(nf_operator *op, const float2 *vg, int B, int b, float *wpart, float *gpart,
                         float *r2_phys, cudaStream_t s) {
    const nf_kernel &k = op->kp;
    const float k2 = (k.s1 * k.s1) / (k.s2 * k.s2);
    const int m = adj_form(k);
    const double L2E = 1.4426950408889634;
    *r2_phys = (float)((m > 0 ? (double)k.s2 * k.s2 : (double)k.s1 * k.s1) / L2E);
    const bool cull = op->mf_cull && op->adj_pairs;
    const int blk = adj_block(op);
    dim3 grid((unsigned)(cull ? op->adj_live : sym_pair_count(op)), 1, 1);
    const size_t smem = as_smem_floats(blk) * sizeof(float);
#define NF_ADJ_ARGS                                                                                       \
    op->xyz, vg, op->rowperm, op->n_pad, B, b, k2, k.A1, k.A2, scaled_period(k), wpart, gpart, \
        (cull ? op->adj_pairs : nullptr)
#define NF_ADJ_LAUNCH(RR, BB)                                                                     \
    switch (m) {                                                                                  \
        case 2: adj_sym_kernel<RR, 2, BB><<<grid, MS_THREADS, smem, s>>>(NF_ADJ_ARGS); break;     \
        case 3: adj_sym_kernel<RR, 3, BB><<<grid, MS_THREADS, smem, s>>>(NF_ADJ_ARGS); break;     \
        case 4: adj_sym_kernel<RR, 4, BB><<<grid, MS_THREADS, smem, s>>>(NF_ADJ_ARGS); break;     \
        default: adj_sym_kernel<RR, 0, BB><<<grid, MS_THREADS, smem, s>>>(NF_ADJ_ARGS); break;    \
    }
    if (blk == 512) {
        if (op->adj_r == 8) {
            NF_ADJ_LAUNCH(8, 512)
        } else {
            NF_ADJ_LAUNCH(4, 512)
        }
    } else {
        if (op->adj_r == 8) {
            NF_ADJ_LAUNCH(8, 1024)
        } else {
            NF_ADJ_LAUNCH(4, 1024)
        }
    }
#undef NF_ADJ_LAUNCH
#undef NF_ADJ_ARGS
    NF_CUDA_TRY(cudaGetLastError());
    return NF_OK;
}

// Shape of the adjoint pair kernel -- rows per warp (4: two CTAs per SM; 8: one CTA per SM)
// and node block (1,024, or 512 where the 1,024-node block pairs fill fewer than eight waves
// of CTAs) -- chosen by timing the candidates on the operator's own node set: three launches
// each, each between its own events; the fastest of the last two counts.  The launches write
// the call's scratch buffers only (sized for 512-node blocks), before the call's own passes
// overwrite them.
nf_status adj_autotune(nf_operator *op, const float2 *vg, int B, float *wpart, float *gpart, cudaStream_t s) {
    if (op->adj_r) return NF_OK;
    // 512-node blocks only on the automatic schedule without culling: an explicit symmetric
    // schedule pins the block size, and the culled pass's live-pair lists use 1,024-node
    // blocks.  The choice is cached per (device, node count, kernel form, whether 512 is
    // allowed), so operators on the same node set run the same shape (culled and unculled
    // gradients then agree bit for bit).
    static std::mutex mu;
    static std::map<std::tuple<int, int64_t, int, bool>, std::pair<int, int>> cache;
    const bool cull = op->mf_cull && op->adj_pairs;
    const bool try512 = !cull && op->mf_sched == NF_MF_AUTO && sym_pairs_1024(op) < 8 * (int64_t)num_sms();
    const auto key = std::make_tuple(op->device, op->n_pad, adj_form(op->kp), try512);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            op->adj_r = it->second.first;
            op->adj_blk = it->second.second;
            return NF_OK;
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    NF_CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ce, "cudaEventCreate", __FILE__, __LINE__);
    }
    const int cand_r[4] = {4, 8, 4, 8}, cand_b[4] = {1024, 1024, 512, 512};
    float best = 3.4e38f;
    int best_r = 4, best_b = 1024;
    nf_status st = NF_OK;
    float r2 = 1.f;
    for (int c = 0; c < (try512 ? 4 : 2) && st == NF_OK; ++c) {
        op->adj_r = cand_r[c];
        op->adj_blk = cand_b[c];
        for (int rep = 0; rep < 3 && st == NF_OK; ++rep) {
            ce = cudaEventRecord(e0, s);
            if (ce == cudaSuccess) st = launch_adj_sym(op, vg, B, 0, wpart, gpart, &r2, s);
            if (st == NF_OK && ce == cudaSuccess) ce = cudaEventRecord(e1, s);
            if (st == NF_OK && ce == cudaSuccess) ce = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (st == NF_OK && ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
            if (ce != cudaSuccess && st == NF_OK) st = cuda_fail(ce, "adjoint autotune", __FILE__, __LINE__);
            if (st == NF_OK && rep >= 1 && ms < best) {  // the first launch warms up
                best = ms;
                best_r = cand_r[c];
                best_b = cand_b[c];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    op->adj_r = st == NF_OK ? best_r : 0;
    op->adj_blk = st == NF_OK ? best_b : 0;
    if (st == NF_OK) {
        std::lock_guard<std::mutex> lock(mu);
        cache[key] = {best_r, best_b};
    }
    return st;
}

int mf_splits(nf_operator *op, int B) {
    return (B <= kSymMaxB && use_sym(op)) ? sym_slots(op) : mf_plan(op).splits;
}

static SplitPlan variant_plan(int64_t n_pad, int v) {
    return plan_splits(n_pad, MF_WARPS * kMfVariants[v].R, kMfVariants[v].TJ, variant_resident(v));
}

SplitPlan mf_plan(nf_operator *op) {
    if (op->mf_variant < 0) op->mf_variant = default_variant(op->n_pad);
    return variant_plan(op->n_pad, op->mf_variant);
}

// Shape of the single-trajectory (symmetric) launch: rows per warp, block width, slots.
void mf_launch_shape(nf_operator *op, int *R, int *TJ, int *splits) {
    if (!use_sym(op)) {
        const SplitPlan pl = mf_plan(op);
        *R = kMfVariants[op->mf_variant].R;
        *TJ = kMfVariants[op->mf_variant].TJ;
        *splits = pl.splits;
        return;
    }
    *R = op->mf_sym_r;
    *TJ = op->sym_blk;
    *splits = sym_slots(op);
}

// Rows per warp of the scalar multi-trajectory kernel (2 or 4 are instantiated).
static int mf_rows_per_warp(int64_t n_pad) { return n_pad >= 16384 ? 4 : 2; }

// Time the symmetric kernel's launch shapes (rows per warp 4 or 8) once on this operator's
// size and keep the fastest (cached per device, padded size and width ratio).  Runs
// outside any stream capture.
nf_status mf_autotune(nf_operator *op, cudaStream_t s) {
    static std::mutex mu;
    static std::map<std::tuple<int, int64_t, int>, std::pair<int, int>> cache;
    op->mf_variant = default_variant(op->n_pad);
    if (3 * sym_pairs_1024(op) < 2 * (int64_t)num_sms() || !sym_layout_fits(op))
        return NF_OK;  // packed by default
    const auto key = std::make_tuple(op->device, op->n_pad, sym_form(op->kp));
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            op->mf_sym_r = it->second.first;
            op->sym_blk = it->second.second;
            return NF_OK;
        }
    }
    cudaEvent_t e0, e1;
    NF_CUDA_TRY(cudaEventCreate(&e0));
    NF_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_r = 8, best_blk = 1024;
    // (rows per warp, block size): 512-node blocks only where 1,024-node pairs fill fewer than
    // four waves of two CTAs per SM (n below ~49,000); measured on GB300 they win on small
    // sets (n = 20,000: 0.177 vs 0.198 ms) and lose badly on large ones (n = 1e5: 7.2 vs 1.8 ms)
    const bool try512 = sym_pairs_1024(op) < 8 * (int64_t)num_sms();
    NF_TRY(ensure_workspace(op, 1, (int)(op->n_pad / (try512 ? 512 : MS_BLK))));
    NF_CUDA_TRY(cudaMemsetAsync(op->g, 0, sizeof(float) * op->n_pad, s));
    const std::pair<int, int> shapes[3] = {{4, 1024}, {8, 1024}, {8, 512}};
    for (const auto &sh : shapes) {
        if (sh.second == 512 && !try512) continue;
        op->mf_sym_r = sh.first;
        op->sym_blk = sh.second;
        NF_TRY(launch_sym(op, 1, 0, s));  // warm-up
        // each launch between its own events, the fastest of three: host-side gaps between
        // launches (a profiler attached to the process, a busy host) then do not enter
        float ms = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            NF_CUDA_TRY(cudaEventRecord(e0, s));
            NF_TRY(launch_sym(op, 1, 0, s));
            NF_CUDA_TRY(cudaEventRecord(e1, s));
            NF_CUDA_TRY(cudaEventSynchronize(e1));
            float t = 0.f;
            NF_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
            ms = std::min(ms, t);
        }
        if (ms < best) {
            best = ms;
            best_r = sh.first;
            best_blk = sh.second;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    op->mf_sym_r = best_r;
    op->sym_blk = best_blk;
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = {best_r, best_blk};
    return NF_OK;
}

// ---- block-pair culling (opt-in).  A block pair whose bounding boxes are so far apart that
// the wider Gaussian's exponent exceeds 160 (log2 units) for every pair in it contributes
// exactly zero in FP32: ex2 flushes results below 2^-126 to 0, e1 = e2^m then is 0 too, and
// adding those zeros leaves every row and column sum unchanged.  Culling skips such pairs:
// the symmetric kernel runs over the live pairs only, and each node then adds the slots of
// its block's live pairs, in ascending slot order, into slot 0 -- the same nonzero terms in
// the same order as the full sum, so results are bit-identical to it.
__global__ void cull_reduce_kernel(float *__restrict__ partial, int64_t n_pad, int B, int b0,
                                   const int *__restrict__ node_blk, const int *__restrict__ ptr,
                                   const int *__restrict__ slots) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = b0 + blockIdx.y;  // trajectory
    if (i >= n_pad) return;
    const int K = node_blk[i];
    float acc = 0.f;
    for (int p = ptr[K]; p < ptr[K + 1]; ++p) acc += partial[((int64_t)slots[p] * B + b) * n_pad + i];
    partial[(int64_t)b * n_pad + i] = acc;
}

// The adjoint pass over culled pairs: each node adds its 1,024-node block's live W nu slots
// of trajectory b into slot 0 (the epilogue then reads one slot).
nf_status launch_adj_cull_reduce(nf_operator *op, float *wpart, int B, int b, cudaStream_t s) {
    cull_reduce_kernel<<<dim3((unsigned)ceil_div(op->n_pad, 256), 1), 256, 0, s>>>(
        wpart, op->n_pad, B, b, op->adj_node_blk, op->adj_ptr, op->adj_slots);
    NF_CUDA_TRY(cudaGetLastError());
    return NF_OK;
}

// Live block pairs of the node blocks of size blk (Morton order), in coordinates scaled by sk
// from the stored s1 units, for a kernel whose wider exponential has exponent wide * r^2
// there; per: the period in s1 units (0: none).  Also each block's live slots (CSR) and each
// node's block.
struct CullLists {
    std::vector<int> pairs, ptr, slots, node_blk;
};

static void build_cull_lists(const std::vector<float> &xyz, const std::vector<int> &perm, int64_t n, int64_t n_pad,
                             int64_t blk, double sk, double wide, double per, CullLists &L) {
    const int64_t nb = n_pad / blk, npairs = nb * (nb + 1) / 2;
    std::vector<double> lo((size_t)3 * nb, 1e300), hi((size_t)3 * nb, -1e300);
    std::vector<char> empty((size_t)nb, 1);
    L.node_blk.assign((size_t)n_pad, 0);
    for (int64_t p = 0; p < n_pad; ++p) {
        const int node = perm[(size_t)p];
        const int64_t K = p / blk;
        L.node_blk[(size_t)node] = (int)K;
        if (node >= n) continue;
        empty[(size_t)K] = 0;
        for (int d = 0; d < 3; ++d) {
            const double v = (double)xyz[(size_t)d * n_pad + node] * sk;
            lo[(size_t)(3 * K + d)] = std::min(lo[(size_t)(3 * K + d)], v);
            hi[(size_t)(3 * K + d)] = std::max(hi[(size_t)(3 * K + d)], v);
        }
    }
    const double pers = per * sk;
    auto live = [&](int64_t I, int64_t J) {
        if (I == J) return true;
        if (empty[(size_t)I] || empty[(size_t)J]) return false;  // no real node: all g are 0
        double d2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double cI = 0.5 * (lo[(size_t)(3 * I + d)] + hi[(size_t)(3 * I + d)]);
            const double cJ = 0.5 * (lo[(size_t)(3 * J + d)] + hi[(size_t)(3 * J + d)]);
            const double H = 0.5 * (hi[(size_t)(3 * I + d)] - lo[(size_t)(3 * I + d)]) +
                             0.5 * (hi[(size_t)(3 * J + d)] - lo[(size_t)(3 * J + d)]);
            double D = cJ - cI;
            if (pers > 0.0 && d < 2) D -= pers * std::nearbyint(D / pers);  // nearest image
            const double gap = std::max(0.0, std::fabs(D) - H);
            d2 += gap * gap;
        }
        return wide * d2 < 160.0 * (1.0 + 1e-4);
    };
    std::vector<char> lv((size_t)npairs);
    L.pairs.clear();
    for (int64_t J = 0; J < nb; ++J)
        for (int64_t I = 0; I <= J; ++I) {
            const int64_t t = J * (J + 1) / 2 + I;
            lv[(size_t)t] = live(I, J) ? 1 : 0;
            if (lv[(size_t)t]) L.pairs.push_back((int)t);
        }
    L.ptr.assign((size_t)nb + 1, 0);
    L.slots.clear();
    for (int64_t K = 0; K < nb; ++K) {
        for (int64_t S = 0; S < nb; ++S) {
            const int64_t a = std::min(K, S), b = std::max(K, S);
            if (lv[(size_t)(b * (b + 1) / 2 + a)]) L.slots.push_back((int)S);
        }
        L.ptr[(size_t)K + 1] = (int)L.slots.size();
    }
}

static nf_status upload_int(const std::vector<int> &v, int **dst, cudaStream_t s) {
    cudaFree(*dst);
    *dst = nullptr;
    NF_CUDA_TRY(cudaMalloc(dst, sizeof(int) * std::max<size_t>(1, v.size())));
    NF_CUDA_TRY(cudaMemcpyAsync(*dst, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice, s));
    return NF_OK;
}

nf_status mf_set_cull(nf_operator *op, int enable, int64_t *live_out, int64_t *total_out, cudaStream_t s) {
    const int64_t n = op->n, n_pad = op->n_pad, blk = op->sym_blk, nb = n_pad / blk, npairs = nb * (nb + 1) / 2;
    if (total_out) *total_out = npairs;
    if (live_out) *live_out = npairs;
    if (op->mf_cull) destroy_graphs(op);
    op->mf_cull = 0;
    if (!enable) return NF_OK;
    // boxes of the Morton blocks over their real nodes, in the kernels' coordinate units
    std::vector<float> xyz((size_t)3 * n_pad);
    std::vector<int> perm((size_t)n_pad);
    NF_CUDA_TRY(cudaMemcpyAsync(xyz.data(), op->xyz, sizeof(float) * 3 * n_pad, cudaMemcpyDeviceToHost, s));
    NF_CUDA_TRY(cudaMemcpyAsync(perm.data(), op->rowperm, sizeof(int) * n_pad, cudaMemcpyDeviceToHost, s));
    NF_CUDA_TRY(cudaStreamSynchronize(s));
    const nf_kernel &k = op->kp;
    const int form = sym_form(k);
    const double k2 = ((double)k.s1 * k.s1) / ((double)k.s2 * k.s2);
    const double per = (double)scaled_period(k);
    // forward: the symmetric kernel's units (s2 when m >= 2) and its wider exponential
    // (the second Gaussian is not evaluated when A2 = 0)
    CullLists fw, ad;
    build_cull_lists(xyz, perm, n, n_pad, blk, form >= 2 ? std::sqrt(k2) : 1.0,
                     form > 0 ? 1.0 : std::min(1.0, k2), per, fw);
    // adjoint: 1,024-node blocks, and both Gaussians always (the parameter sums of A2 and s2
    // need e2 even when A2 = 0)
    build_cull_lists(xyz, perm, n, n_pad, MS_BLK, 1.0, std::min(1.0, k2), per, ad);
    NF_TRY(upload_int(fw.pairs, &op->cull_pairs, s));
    NF_TRY(upload_int(fw.ptr, &op->cull_ptr, s));
    NF_TRY(upload_int(fw.slots, &op->cull_slots, s));
    NF_TRY(upload_int(fw.node_blk, &op->node_blk, s));
    NF_TRY(upload_int(ad.pairs, &op->adj_pairs, s));
    NF_TRY(upload_int(ad.ptr, &op->adj_ptr, s));
    NF_TRY(upload_int(ad.slots, &op->adj_slots, s));
    NF_TRY(upload_int(ad.node_blk, &op->adj_node_blk, s));
    NF_CUDA_TRY(cudaStreamSynchronize(s));
    op->cull_live = (int64_t)fw.pairs.size();
    op->adj_live = (int64_t)ad.pairs.size();
    op->mf_cull = 1;
    if (live_out) *live_out = op->cull_live;
    return NF_OK;
}

nf_status launch_mf_pair(nf_operator *op, int B, cudaStream_t s, int *splits_out) {
    if (B <= kSymMaxB && use_sym(op)) {  // symmetric kernel, one partial slot per node block
        NF_TRY(launch_sym(op, B, 0, s));
        *splits_out = sym_slots(op);
        if (op->mf_cull) {  // only live pairs ran: add each node's live slots into slot 0
            cull_reduce_kernel<<<dim3((unsigned)ceil_div(op->n_pad, 256), (unsigned)B), 256, 0, s>>>(
                op->partial, op->n_pad, B, 0, op->node_blk, op->cull_ptr, op->cull_slots);
            NF_CUDA_TRY(cudaGetLastError());
            *splits_out = 1;
        }
        return NF_OK;
    }
    if (B == 1) {  // a small node set: the packed kernel over (row block, column split) items
        const SplitPlan pl = mf_plan(op);
        NF_TRY(launch_mf_packed(op, 1, 0, 1, pl, s));
        *splits_out = pl.splits;
        return NF_OK;
    }
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
                case 16: st = launch_mf_group<16, 4>(op, B, b, groups, spl, s); break;
                case 8: st = launch_mf_group<8, 4>(op, B, b, groups, spl, s); break;
                case 4: st = launch_mf_group<4, 4>(op, B, b, groups, spl, s); break;
                default: st = launch_mf_group<2, 4>(op, B, b, groups, spl, s); break;
            }
        } else {
            switch (nb) {
                case 16: st = launch_mf_group<16, 2>(op, B, b, groups, spl, s); break;
                case 8: st = launch_mf_group<8, 2>(op, B, b, groups, spl, s); break;
                case 4: st = launch_mf_group<4, 2>(op, B, b, groups, spl, s); break;
                default: st = launch_mf_group<2, 2>(op, B, b, groups, spl, s); break;
            }
        }
        b += groups * nb;
        return st;
    };
    NF_TRY(run(16));
    NF_TRY(run(8));
    NF_TRY(run(4));
    NF_TRY(run(2));
    NF_TRY(run(1));
    *splits_out = pl.splits;
    return NF_OK;
}

// Launch plan of launch_mf_pair_single: at most max_splits column splits.
SplitPlan plan_mf_pair_single(int64_t n_pad, int max_splits) {
    const int R = mf_rows_per_warp(n_pad);
    return plan_splits(n_pad, MF_WARPS * R, MF_TJ, R == 4 ? mf_resident<1, 4>() : mf_resident<1, 2>(), max_splits);
}

// Single-trajectory pair sums into caller-provided buffers (x4, g padded to n_pad,
// partial [splits][n_pad]); the planner considers at most max_splits column splits.
nf_status launch_mf_pair_single(const float4 *x4, const float *g, int64_t n_pad, const nf_kernel &k, int max_splits,
                                float *partial, int *err, cudaStream_t s, int *splits_out) {
    const int R = mf_rows_per_warp(n_pad);
    const SplitPlan pl = plan_mf_pair_single(n_pad, max_splits);
    const float L2E = 1.4426950408889634f;
    const float c1 = -L2E / (k.s1 * k.s1), c2 = -L2E / (k.s2 * k.s2);
    dim3 grid((unsigned)pl.row_blocks, (unsigned)pl.splits, 1);
    if (R == 4)
        mf_pair_kernel<1, 4><<<grid, MF_THREADS, sizeof(MfSmem<1>), s>>>(x4, g, n_pad, 1, 0, pl.jchunk, c1, c2, k.A1,
                                                                      k.A2, k.period, partial, err);
    else
        mf_pair_kernel<1, 2><<<grid, MF_THREADS, sizeof(MfSmem<1>), s>>>(x4, g, n_pad, 1, 0, pl.jchunk, c1, c2, k.A1,
                                                                      k.A2, k.period, partial, err);
    NF_CUDA_TRY(cudaGetLastError());
    *splits_out = pl.splits;
    return NF_OK;
}

// ----------------------------------------------------------------------------
// Row order of the packed pair kernel: nodes sorted by the Morton (Z-order) code of their
// cell in a 1024^3 grid over the bounding box, ties by index, so that consecutive rows --
// the R rows of a warp -- are near each other.  Keys (code << 32 | index) are unique; a
// bitonic network over the next power of two sorts them.  Padding rows keep their place.

// Bounding box of the first n coordinates (one block): box = {lo x, lo y, lo z, hi x, hi y, hi z}.
__global__ void row_bbox_kernel(const float *__restrict__ xyz, int64_t n, int64_t n_pad, float *__restrict__ box) {
    __shared__ float red[6][32];
    float v[6] = {3.4e38f, 3.4e38f, 3.4e38f, -3.4e38f, -3.4e38f, -3.4e38f};
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
        for (int d = 0; d < 3; ++d) {
            const float c = xyz[d * n_pad + j];
            v[d] = fminf(v[d], c);
            v[3 + d] = fmaxf(v[3 + d], c);
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1)
        for (int d = 0; d < 3; ++d) {
            v[d] = fminf(v[d], __shfl_xor_sync(0xffffffffu, v[d], o));
            v[3 + d] = fmaxf(v[3 + d], __shfl_xor_sync(0xffffffffu, v[3 + d], o));
        }
    if (lane == 0)
        for (int d = 0; d < 6; ++d) red[d][warp] = v[d];
    __syncthreads();
    if (threadIdx.x < 6) {
        const int d = threadIdx.x;
        float a = red[d][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) a = d < 3 ? fminf(a, red[d][w]) : fmaxf(a, red[d][w]);
        box[d] = a;
    }
}

// 10 bits of v spread to every third bit position.
__device__ __forceinline__ uint32_t spread_bits3(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void row_key_kernel(const float *__restrict__ xyz, int64_t n, int64_t n_pad, int64_t m,
                               const float *__restrict__ box, unsigned long long *__restrict__ keys) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    if (j >= n) {
        keys[j] = ~0ull;
        return;
    }
    uint32_t code = 0;
    for (int d = 0; d < 3; ++d) {
        const float ext = box[3 + d] - box[d];
        const float t = ext > 0.f ? (xyz[d * n_pad + j] - box[d]) / ext : 0.f;
        const uint32_t c = (uint32_t)fminf(fmaxf(t * 1024.f, 0.f), 1023.f);
        code |= spread_bits3(c) << d;
    }
    keys[j] = ((unsigned long long)code << 32) | (unsigned long long)j;
}

// One compare-exchange step of the bitonic network (block size kk, partner distance jj).
__global__ void row_bitonic_kernel(unsigned long long *__restrict__ keys, int64_t m, int64_t jj, int64_t kk) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int64_t l = i ^ jj;
    if (l <= i) return;
    const unsigned long long a = keys[i], b = keys[l];
    const bool ascending = (i & kk) == 0;
    if ((a > b) == ascending) {
        keys[i] = b;
        keys[l] = a;
    }
}

__global__ void row_perm_kernel(const unsigned long long *__restrict__ keys, int64_t n, int64_t n_pad,
                                int *__restrict__ rowperm) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_pad) return;
    rowperm[k] = k < n ? (int)(keys[k] & 0xffffffffull) : (int)k;
}

nf_status mf_build_row_order(nf_operator *op, cudaStream_t s) {
    const int64_t n = op->n, n_pad = op->n_pad;
    int64_t m = 1;
    while (m < n_pad) m <<= 1;
    NF_CUDA_TRY(cudaMalloc(&op->rowperm, sizeof(int) * n_pad));
    unsigned long long *keys = nullptr;
    float *box = nullptr;
    NF_CUDA_TRY(cudaMalloc(&keys, sizeof(unsigned long long) * m + 64));
    box = reinterpret_cast<float *>(keys + m);
    nf_status st = NF_OK;
    row_bbox_kernel<<<1, 1024, 0, s>>>(op->xyz, n, n_pad, box);
    row_key_kernel<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(op->xyz, n, n_pad, m, box, keys);
    for (int64_t kk = 2; kk <= m; kk <<= 1)
        for (int64_t jj = kk >> 1; jj > 0; jj >>= 1)
            row_bitonic_kernel<<<(unsigned)ceil_div(m, 256), 256, 0, s>>>(keys, m, jj, kk);
    row_perm_kernel<<<(unsigned)ceil_div(n_pad, 256), 256, 0, s>>>(keys, n, n_pad, op->rowperm);
    float hbox[6] = {0, 0, 0, 0, 0, 0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hbox, box, sizeof(hbox), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    op->planar = (e == cudaSuccess && hbox[2] == hbox[5]) ? 1 : 0;  // one z for every node
    if (e != cudaSuccess) st = cuda_fail(e, "row order", __FILE__, __LINE__);
    cudaFree(keys);
    return st;
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
    const bool mf = q_on_vector(op);
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
    const float acc = sum_slots(partial + (int64_t)b * n_pad + i, (int64_t)B * n_pad, splits);
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
    const float4 *x4;   // node coordinates (the flat manufactured forcing)
    nf_kernel kp;
    const double *t0;
    double dt;
    int stage;
    long long *step_ctr;
    unsigned *done_ctr;
    float *ckpt;
    int C;
    int *err;           // operator's device flag: DEV_NONFINITE on a non-finite new state
};

// Flat manufactured forcing (NF_FORCE_MMS_FLAT).  One factor of the convolution term:
//   J(a) = int_{-L/2}^{L/2} exp(-p d^2) exp(-e(d)^2 / (2 sigma^2)) dd,  e(d) = nearest image of a - d,
// a = nearest image of x - x0 in one coordinate.  e(d) = a - d except past the point where
// a - d leaves [-L/2, L/2] (d < a - L/2 for a >= 0, d > a + L/2 for a < 0), where it is
// a - d -+ L.  Each piece is a Gaussian product integrated in closed form:
//   int_{d0}^{d1} exp(-p d^2 - r (d - a')^2) dd
//     = exp(-p r a'^2 / (p + r)) (1/2) sqrt(pi / (p + r)) [erf(k (d1 - m)) - erf(k (d0 - m))],
// r = 1 / (2 sigma^2), m = r a' / (p + r), k = sqrt(p + r).
constexpr double kPi = 3.14159265358979323846;
__device__ __forceinline__ double gauss_piece(double p, double r, double a, double d0, double d1) {
    const double s = p + r, m = r * a / s, k = sqrt(s);
    return exp(-p * r * a * a / s) * 0.5 * sqrt(kPi / s) * (erf(k * (d1 - m)) - erf(k * (d0 - m)));
}
__device__ __forceinline__ double flat_factor(double a, double p, double r, double L) {
    const double h = 0.5 * L;
    if (a >= 0.0) return gauss_piece(p, r, a - L, -h, a - h) + gauss_piece(p, r, a, a - h, h);
    return gauss_piece(p, r, a, -h, a + h) + gauss_piece(p, r, a + L, a + h, h);
}
__device__ __forceinline__ double nearest_image(double d, double L) { return d - L * rint(d / L); }

__device__ __forceinline__ double forcing_value(const nf_forcing &F, const float4 *x4, const nf_kernel &kp,
                                                int64_t i, double t, float beta, float theta) {
    if (F.kind == NF_FORCE_MMS_FLAT) {
        // z = G(x, x0(t); sigma) + c on the periodic square; gamma = du*/dt + u* - scale C,
        // C = int_cell w(dist(x, y)) z(y) dy: the constant part integrates w over the
        // displacement square, the Gaussian part is separable (flat_factor per coordinate)
        const double L = kp.period, sg = F.sigma, r = 1.0 / (2.0 * sg * sg);
        const double x0 = F.radius * cos(t), y0 = F.radius * sin(t);
        const float4 xi = x4[i];
        const double ax = nearest_image((double)xi.x - x0, L), ay = nearest_image((double)xi.y - y0, L);
        const double G = exp(-(ax * ax + ay * ay) * r) / (2.0 * kPi * sg * sg);
        const double z = G + F.c;
        const double dz = G * (ax * (-F.radius * sin(t)) + ay * (F.radius * cos(t))) / (sg * sg);
        const double us = (double)theta + log(z / (1.0 - z)) / (double)beta;
        const double dus = dz / ((double)beta * z * (1.0 - z));
        const double amp[2] = {(double)kp.A1, -(double)kp.A2}, wid[2] = {(double)kp.s1, (double)kp.s2};
        double C = 0.0;
        for (int h = 0; h < 2; ++h) {
            if (amp[h] == 0.0) continue;
            const double p = 1.0 / (wid[h] * wid[h]);
            const double e = sqrt(kPi) * wid[h] * erf(0.5 * L / wid[h]);
            C += amp[h] * (F.c * e * e + flat_factor(ax, p, r, L) * flat_factor(ay, p, r, L) /
                                             (2.0 * kPi * sg * sg));
        }
        return dus + us - F.scale * C;
    }
    if (F.kind != NF_FORCE_MMS_EIGEN && F.kind != NF_FORCE_MMS_SPHERE) return 0.0;
    double Y1, Y2;
    if (F.kind == NF_FORCE_MMS_SPHERE) {  // Y1 = z / 2 (degree 1), Y2 = x y (degree 2) at the node
        const float4 xi = x4[i];
        Y1 = 0.5 * (double)xi.z;
        Y2 = (double)xi.x * (double)xi.y;
    } else {
        Y1 = F.Y1[i];
        Y2 = F.Y2[i];
    }
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
        float I = sum_slots(a.partial + (int64_t)b * a.n_pad + i, (int64_t)a.B * a.n_pad, a.splits);
        if (a.rs) I *= a.rs[i];
        const double cs = (a.stage == 1) ? 0.0 : (a.stage == 4 ? 1.0 : 0.5);
        const double ts = *a.t0 + (double)step * a.dt + cs * a.dt;
        const float bb = a.beta[b], th = a.theta[b];
        const float gam = (float)forcing_value(a.F, a.x4, a.kp, i, ts, bb, th);
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
            if (!isfinite(unew) && *a.err == DEV_OK) atomicCAS(a.err, DEV_OK, DEV_NONFINITE);
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
    a.q = q_on_vector(op) ? op->q : nullptr;
    a.rs = (op->path == NF_DENSE_BF16X2) ? op->rs : nullptr;
    a.beta = p.beta;
    a.theta = p.theta;
    a.F = p.forcing;
    a.x4 = op->x4;
    a.kp = op->kp;
    a.t0 = op->t0_dev;
    a.dt = p.dt;
    a.stage = p.stage;
    a.step_ctr = op->step_ctr;
    a.done_ctr = op->done_ctr;
    a.ckpt = p.ckpt;
    a.C = p.C;
    a.err = op->err;
    const int64_t tot = (int64_t)B * op->n;
    const int T = 256;
    rk4_stage_kernel<<<(unsigned)ceil_div(tot, T), T, 0, s>>>(a);
    NF_CUDA_TRY(cudaGetLastError());
    return NF_OK;
}

}  // namespace nfi
