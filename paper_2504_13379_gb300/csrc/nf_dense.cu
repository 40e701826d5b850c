// nf_dense.cu -- precomputed operator W diag(q) of Eq. (2.9) and its streaming
// matrix-vector product.
//
// Build (once per operator): WQ[i, j] = w(|x_i - x_j|) q_j, row-major, leading
// dimension n_pad (padded columns are zero because q is zero there).
//   NF_DENSE_FP32:   FP32 plane.
//   NF_DENSE_BF16X2: s_i = 2^ceil(log2 max_j |WQ_ij|) (a power of two, so dividing by
//                    it is exact); hi = bf16_rn(WQ/s_i), lo = bf16_rn(WQ/s_i - hi).
//                    hi + lo carries ~16 significant bits; I_i = s_i sum_j (hi+lo) F_j.
//                    The two planes use the blocked layout (128 x 64 blocks of 16 KB), the
//                    tile the batched tensor-core GEMM reads with one sequential copy.
// Apply (every stage): HBM-bound stream of 4 bytes per entry for either plane type.
//   NF_DENSE_SYM_FP32: the kernel matrix K_ij = w(|x_i - x_j|) itself (q moves to the vector
//                    side, g = q o f), symmetric, so only its upper-triangle 1024 x 1024
//                    blocks are stored (n_pad^2 / 2 + n_pad * 512 entries).  One CTA streams
//                    a block (I <= J) once and produces both its row sums (K_IJ g_J, to
//                    partial slot J) and its column sums (K_IJ^T g_I, to slot I): half the
//                    HBM bytes of the full matrix per stage.
//   NF_DENSE_SYM_BF16X2: the same blocks as bf16 hi + lo planes with symmetric power-of-two
//                    scaling s_i s_j (the vector is scaled on the way in, each output by its
//                    own s_i): the precision form of the symmetric operator.
// Work items (32-row block, column split) write partial sums like the matrix-free
// kernel, so the same stage kernel finishes the RK4 step.
#include "nf_internal.cuh"

#include <algorithm>

namespace nfi {

// ---------------------------------------------------------------- build
__device__ __forceinline__ float mexhat(float r2, float A1, float is1, float A2, float is2) {
    return A1 * expf(-r2 * is1) - A2 * expf(-r2 * is2);
}

// Squared distance; per > 0: x and y differences reduced to their nearest images (§4,
// Eq. (dist)), ip = 1 / per.
__device__ __forceinline__ float pair_r2(float4 a, float4 b, float per, float ip) {
    float dx = a.x - b.x, dy = a.y - b.y;
    const float dz = a.z - b.z;
    if (per > 0.f) {
        dx = wrap1(dx, per, ip);
        dy = wrap1(dy, per, ip);
    }
    return dx * dx + dy * dy + dz * dz;
}

// one block per row i; FP32 plane
__global__ void dense_build_fp32_kernel(const float4 *__restrict__ x4, const float *__restrict__ q, int64_t n,
                                        int64_t n_pad, float A1, float is1, float A2, float is2, float per,
                                        float ip, float *__restrict__ W) {
    const int64_t i = blockIdx.x;
    const float4 xi = x4[i];
    float *row = W + i * n_pad;
    for (int64_t j = threadIdx.x; j < n_pad; j += blockDim.x) {
        const float4 xj = x4[j];
        const float r2 = pair_r2(xi, xj, per, ip);
        row[j] = mexhat(r2, A1, is1, A2, is2) * q[j];
    }
}

// one block per row: row scale s_i (power of two), then hi / lo planes
__global__ void dense_build_bf16x2_kernel(const float4 *__restrict__ x4, const float *__restrict__ q, int64_t n,
                                          int64_t n_pad, float A1, float is1, float A2, float is2, float per,
                                          float ip, uint16_t *__restrict__ Whi, uint16_t *__restrict__ Wlo,
                                          float *__restrict__ rs) {
    __shared__ float red[32];
    const int64_t i = blockIdx.x;
    const float4 xi = x4[i];
    float mx = 0.f;
    for (int64_t j = threadIdx.x; j < n_pad; j += blockDim.x) {
        const float4 xj = x4[j];
        const float r2 = pair_r2(xi, xj, per, ip);
        mx = fmaxf(mx, fabsf(mexhat(r2, A1, is1, A2, is2) * q[j]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    mx = red[0];
    // s = 2^e with mx <= s (frexp: mx = m 2^e, m in [0.5, 1))
    int e = 0;
    float s = 1.f;
    if (mx > 0.f) {
        (void)frexpf(mx, &e);
        s = ldexpf(1.f, e);
    }
    const float inv = 1.f / s;  // exact: power of two
    if (threadIdx.x == 0) rs[i] = s;
    for (int64_t j = threadIdx.x; j < n_pad; j += blockDim.x) {
        const float4 xj = x4[j];
        const float r2 = pair_r2(xi, xj, per, ip);
        const float v = mexhat(r2, A1, is1, A2, is2) * q[j] * inv;
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        const int64_t o = blocked_offset(i, j, n_pad);
        Whi[o] = __bfloat16_as_ushort(hi);
        Wlo[o] = __bfloat16_as_ushort(lo);
    }
}

// ---- symmetric blocks: block pair t = J (J + 1) / 2 + I (I <= J) holds K over rows of node
// block I and columns of node block J, row-major, SB x SB
constexpr int SB = 1024;
constexpr int SYM_THREADS = 256;
constexpr int SYM_WARPS = SYM_THREADS / 32;

__device__ __forceinline__ void sym_block_pair(int64_t t, int &I, int &J) {
    int64_t j = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (j * (j + 1) / 2 > t) --j;
    while ((j + 1) * (j + 2) / 2 <= t) ++j;
    J = (int)j;
    I = (int)(t - j * (j + 1) / 2);
}

// grid (pairs, SB / 16): each block writes 16 rows of one block pair
__global__ void dense_build_sym_kernel(const float4 *__restrict__ x4, float A1, float is1, float A2, float is2,
                                       float per, float ip, float *__restrict__ K) {
    int I, J;
    sym_block_pair(blockIdx.x, I, J);
    float *blk = K + (int64_t)blockIdx.x * SB * SB;
    for (int rr = 0; rr < 16; ++rr) {
        const int r = blockIdx.y * 16 + rr;
        const float4 xi = x4[(int64_t)I * SB + r];
        for (int c = threadIdx.x; c < SB; c += blockDim.x) {
            const float4 xj = x4[(int64_t)J * SB + c];
            const float r2 = pair_r2(xi, xj, per, ip);
            blk[(int64_t)r * SB + c] = mexhat(r2, A1, is1, A2, is2);
        }
    }
}

// ---- symmetric bf16 hi + lo blocks (NF_DENSE_SYM_BF16X2).  K_ij = s_i s_j (hi_ij + lo_ij)
// with s_i = 2^round(log2 sqrt(max_j |K_ij|)) over the real nodes: a power of two, so the
// division by s_i s_j is exact, and the scaled matrix stays symmetric.  hi = bf16_rn(K / s s),
// lo = bf16_rn(K / s s - hi): 16 significant bits, |K / s s - hi - lo| <= 2^-18 |K / s s|.
// Block pair t (I <= J) holds rows of node block I x columns of node block J; a row is 128
// chunks of 8 columns, each chunk 16 bytes of hi followed by 16 bytes of lo (one 32-byte
// piece per lane and chunk).  Entries of padded rows or columns are zero.
constexpr int SBC = SB / 8;  // chunks per block row

__global__ void sym_rowscale_kernel(const float4 *__restrict__ x4, int64_t n, float A1, float is1, float A2,
                                    float is2, float per, float ip, float *__restrict__ sc) {
    __shared__ float red[32];
    const int64_t i = blockIdx.x;
    if (i >= n) {  // padded row: any power of two
        if (threadIdx.x == 0) sc[i] = 1.f;
        return;
    }
    const float4 xi = x4[i];
    float mx = 0.f;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) mx = fmaxf(mx, fabsf(mexhat(pair_r2(xi, x4[j], per, ip), A1, is1, A2, is2)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmaxf(v, red[w]);
        int e = 0;
        if (v > 0.f) {
            (void)frexpf(v, &e);  // v = m 2^e, m in [0.5, 1)
        }
        sc[i] = v > 0.f ? ldexpf(1.f, e / 2) : 1.f;  // ~ sqrt(v), a power of two
    }
}

// grid (pairs, SB / 16): each block writes 16 rows of one block pair
__global__ void dense_build_sym_bf16x2_kernel(const float4 *__restrict__ x4, const float *__restrict__ sc, int64_t n,
                                              float A1, float is1, float A2, float is2, float per, float ip,
                                              uint4 *__restrict__ K) {
    int I, J;
    sym_block_pair(blockIdx.x, I, J);
    uint4 *blk = K + (int64_t)blockIdx.x * SB * SBC * 2;
    for (int rr = 0; rr < 16; ++rr) {
        const int r = blockIdx.y * 16 + rr;
        const int64_t i = (int64_t)I * SB + r;
        const float4 xi = x4[i];
        const float si = sc[i];
        for (int c = threadIdx.x; c < SBC; c += blockDim.x) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                float v[2];
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const int64_t j = (int64_t)J * SB + 8 * c + e + t;
                    v[t] = (i < n && j < n) ? mexhat(pair_r2(xi, x4[j], per, ip), A1, is1, A2, is2) / (si * sc[j]) : 0.f;
                }
                const __nv_bfloat16 h0 = __float2bfloat16_rn(v[0]), h1 = __float2bfloat16_rn(v[1]);
                const __nv_bfloat16 l0 = __float2bfloat16_rn(v[0] - __bfloat162float(h0));
                const __nv_bfloat16 l1 = __float2bfloat16_rn(v[1] - __bfloat162float(h1));
                h[e / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                l[e / 2] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
            }
            blk[((int64_t)r * SBC + c) * 2] = make_uint4(h[0], h[1], h[2], h[3]);
            blk[((int64_t)r * SBC + c) * 2 + 1] = make_uint4(l[0], l[1], l[2], l[3]);
        }
    }
}

nf_status launch_dense_build(nf_operator *op, cudaStream_t s) {
    const nf_kernel &k = op->kp;
    const float is1 = 1.f / (k.s1 * k.s1), is2 = 1.f / (k.s2 * k.s2);
    const float per = k.period > 0.f ? k.period : 0.f, ip = per > 0.f ? 1.f / per : 0.f;
    if (op->path == NF_DENSE_SYM_FP32) {
        const int64_t nb = op->n_pad / SB;
        dense_build_sym_kernel<<<dim3((unsigned)(nb * (nb + 1) / 2), SB / 16), 256, 0, s>>>(op->x4, k.A1, is1, k.A2,
                                                                                       is2, per, ip, op->W32);
    } else if (op->path == NF_DENSE_SYM_BF16X2) {
        const int64_t nb = op->n_pad / SB;
        sym_rowscale_kernel<<<(unsigned)op->n_pad, 256, 0, s>>>(op->x4, op->n, k.A1, is1, k.A2, is2, per, ip, op->rs);
        NF_CUDA_TRY(cudaGetLastError());
        dense_build_sym_bf16x2_kernel<<<dim3((unsigned)(nb * (nb + 1) / 2), SB / 16), 128, 0, s>>>(
            op->x4, op->rs, op->n, k.A1, is1, k.A2, is2, per, ip, reinterpret_cast<uint4 *>(op->Whi));
    } else if (op->path == NF_DENSE_FP32) {
        dense_build_fp32_kernel<<<(unsigned)op->n_pad, 256, 0, s>>>(op->x4, op->q, op->n, op->n_pad, k.A1, is1, k.A2,
                                                               is2, per, ip, op->W32);
    } else {
        dense_build_bf16x2_kernel<<<(unsigned)op->n_pad, 256, 0, s>>>(op->x4, op->q, op->n, op->n_pad, k.A1, is1,
                                                                 k.A2, is2, per, ip, op->Whi, op->Wlo, op->rs);
    }
    NF_CUDA_TRY(cudaGetLastError());
    return NF_OK;
}

// ---------------------------------------------------------------- GEMV
constexpr int DG_THREADS = 256;
constexpr int DG_WARPS = DG_THREADS / 32;
constexpr int DG_R = 4;                        // rows per warp
constexpr int DG_ROWS = DG_WARPS * DG_R;       // rows per block
constexpr int DG_TILE = 1024;                  // columns per inner tile
static_assert(kNodePad % DG_TILE == 0, "tile must divide the node padding");

__device__ __forceinline__ float4 ld_stream_f4(const float *p) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}
__device__ __forceinline__ uint4 ld_stream_u4(const void *p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// FP32 plane.  Lane l of a warp covers columns tile + 4l + 128u, u = 0..7.
__global__ void __launch_bounds__(DG_THREADS)
gemv_fp32_kernel(const float *__restrict__ W, const float *__restrict__ F, int64_t n_pad, int B, int b,
                 int64_t jchunk, float *__restrict__ partial) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int split = blockIdx.y;
    const int64_t row0 = ((int64_t)blockIdx.x * DG_WARPS + warp) * DG_R;
    const int64_t j0 = (int64_t)split * jchunk, j1 = min(n_pad, j0 + jchunk);
    const float *Fb = F + (int64_t)b * n_pad;
    float acc[DG_R] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t t = j0; t < j1; t += DG_TILE) {
#pragma unroll
        for (int uh = 0; uh < 8; uh += 4) {
            float4 w[DG_R][4];
#pragma unroll
            for (int r = 0; r < DG_R; ++r)
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    w[r][u] = ld_stream_f4(W + (row0 + r) * n_pad + t + 128 * (uh + u) + 4 * lane);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 f = __ldg(reinterpret_cast<const float4 *>(Fb + t + 128 * (uh + u) + 4 * lane));
#pragma unroll
                for (int r = 0; r < DG_R; ++r) {
                    acc[r] = fmaf(w[r][u].x, f.x, acc[r]);
                    acc[r] = fmaf(w[r][u].y, f.y, acc[r]);
                    acc[r] = fmaf(w[r][u].z, f.z, acc[r]);
                    acc[r] = fmaf(w[r][u].w, f.w, acc[r]);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < DG_R; ++r) {
        const float v = warp_sum(acc[r]);
        if (lane == 0) partial[((int64_t)split * B + b) * n_pad + row0 + r] = v;
    }
}

// BF16 hi + lo planes.  Lane l covers columns tile + 8l + 256u, u = 0..3.
__global__ void __launch_bounds__(DG_THREADS)
gemv_bf16x2_kernel(const uint16_t *__restrict__ Whi, const uint16_t *__restrict__ Wlo, const float *__restrict__ F,
                   int64_t n_pad, int B, int b, int64_t jchunk, float *__restrict__ partial) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int split = blockIdx.y;
    const int64_t row0 = ((int64_t)blockIdx.x * DG_WARPS + warp) * DG_R;
    const int64_t j0 = (int64_t)split * jchunk, j1 = min(n_pad, j0 + jchunk);
    const float *Fb = F + (int64_t)b * n_pad;
    float acc[DG_R] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t t = j0; t < j1; t += DG_TILE) {
#pragma unroll
        for (int uh = 0; uh < 4; uh += 2) {
            uint4 h[DG_R][2], l[DG_R][2];
#pragma unroll
            for (int r = 0; r < DG_R; ++r)
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int64_t off = blocked_offset(row0 + r, t + 256 * (uh + u) + 8 * lane, n_pad);
                    h[r][u] = ld_stream_u4(Whi + off);
                    l[r][u] = ld_stream_u4(Wlo + off);
                }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float *fp = Fb + t + 256 * (uh + u) + 8 * lane;
                const float4 f0 = __ldg(reinterpret_cast<const float4 *>(fp));
                const float4 f1 = __ldg(reinterpret_cast<const float4 *>(fp + 4));
                const float fv[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
#pragma unroll
                for (int r = 0; r < DG_R; ++r) {
                    const uint32_t hw[4] = {h[r][u].x, h[r][u].y, h[r][u].z, h[r][u].w};
                    const uint32_t lw[4] = {l[r][u].x, l[r][u].y, l[r][u].z, l[r][u].w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float h0 = __uint_as_float(hw[q] << 16), h1 = __uint_as_float(hw[q] & 0xffff0000u);
                        const float l0 = __uint_as_float(lw[q] << 16), l1 = __uint_as_float(lw[q] & 0xffff0000u);
                        acc[r] = fmaf(h0 + l0, fv[2 * q], acc[r]);
                        acc[r] = fmaf(h1 + l1, fv[2 * q + 1], acc[r]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < DG_R; ++r) {
        const float v = warp_sum(acc[r]);
        if (lane == 0) partial[((int64_t)split * B + b) * n_pad + row0 + r] = v;
    }
}

// One CTA per stored block pair (I <= J).  Warp w takes rows w, w + 8, ... of the block;
// lane l covers the columns 4 l + 128 u (u = 0..7) with 16-byte streaming loads.  Row sums:
// dot products with g_J (shared memory), 8 rows at a time reduced across the warp by a
// transposed butterfly; column sums: per lane in registers over the warp's 128 rows,
// then added over the warps in a fixed order.  Diagonal blocks write their row sums only.
__global__ void __launch_bounds__(SYM_THREADS, 2)
gemv_sym_fp32_kernel(const float *__restrict__ K, const float *__restrict__ g_all, int64_t n_pad, int B, int b,
                     float *__restrict__ partial) {
    __shared__ __align__(16) float gI[SB], gJ[SB];
    __shared__ __align__(16) float colred[SYM_WARPS][SB];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int I, J;
    sym_block_pair(blockIdx.x, I, J);
    const bool diag = I == J;
    const float *g = g_all + (int64_t)b * n_pad;
    for (int k = tid; k < SB; k += SYM_THREADS) {
        gI[k] = g[(int64_t)I * SB + k];
        gJ[k] = g[(int64_t)J * SB + k];
    }
    __syncthreads();
    const float *blk = K + (int64_t)blockIdx.x * SB * SB;
    float col[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) col[c] = 0.f;
    float *out_rows = partial + ((int64_t)J * B + b) * n_pad + (int64_t)I * SB;
    for (int r0 = warp; r0 < SB; r0 += 8 * SYM_WARPS) {  // 8 rows per group: r0, r0 + 8, ..., r0 + 56
        float dot[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int r = r0 + 8 * k;
            const float *row = blk + (int64_t)r * SB;
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = ld_stream_f4(row + 4 * lane + 128 * u);
            const float gi = gI[r];
            float d = 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float4 gj = *reinterpret_cast<const float4 *>(gJ + 4 * lane + 128 * u);
                d = fmaf(v[u].x, gj.x, d);
                d = fmaf(v[u].y, gj.y, d);
                d = fmaf(v[u].z, gj.z, d);
                d = fmaf(v[u].w, gj.w, d);
                col[4 * u] = fmaf(v[u].x, gi, col[4 * u]);
                col[4 * u + 1] = fmaf(v[u].y, gi, col[4 * u + 1]);
                col[4 * u + 2] = fmaf(v[u].z, gi, col[4 * u + 2]);
                col[4 * u + 3] = fmaf(v[u].w, gi, col[4 * u + 3]);
            }
            dot[k] = d;
        }
        // transposed butterfly: 7 shuffles reduce the 8 rows' dot products over the warp
        int base = 0, cnt = 8;
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            if (cnt > 1) {
                const int h = cnt >> 1;
                const bool upper = (lane & off) != 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (k < h) {
                        const float send = upper ? dot[k] : dot[k + h];
                        const float keep = upper ? dot[k + h] : dot[k];
                        dot[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                    }
                }
                if (upper) base += h;
                cnt = h;
            } else {
                dot[0] += __shfl_xor_sync(0xffffffffu, dot[0], off);
            }
        }
        if ((lane & 3) == 0) out_rows[r0 + 8 * base] = dot[0];
    }
    if (diag) return;
#pragma unroll
    for (int u = 0; u < 8; ++u)
        *reinterpret_cast<float4 *>(&colred[warp][4 * lane + 128 * u]) =
            make_float4(col[4 * u], col[4 * u + 1], col[4 * u + 2], col[4 * u + 3]);
    __syncthreads();
    float *out_cols = partial + ((int64_t)I * B + b) * n_pad + (int64_t)J * SB;
    for (int k = tid; k < SB; k += SYM_THREADS) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < SYM_WARPS; ++w) v += colred[w][k];
        out_cols[k] = v;
    }
}

// Symmetric bf16 hi + lo blocks: gemv_sym_fp32_kernel's schedule on the scaled planes.  The
// vector is scaled on the way into shared memory (g'_j = s_j g_j) and each output by its own
// s_i, so one stored tile serves I_i = s_i sum_j (hi + lo)_ij g'_j (rows, slot J) and
// I_j = s_j sum_i (hi + lo)_ij g'_i (columns, slot I).  Lane l reads chunks l + 32 u
// (u = 0..3) of a row: 8 columns of hi and of lo, 32 contiguous bytes.
__global__ void __launch_bounds__(SYM_THREADS, 2)
gemv_sym_bf16x2_kernel(const uint4 *__restrict__ K, const float *__restrict__ g_all, const float *__restrict__ sc,
                       int64_t n_pad, int B, int b, float *__restrict__ partial) {
    __shared__ __align__(16) float gI[SB], gJ[SB];
    __shared__ __align__(16) float colred[SYM_WARPS][SB];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int I, J;
    sym_block_pair(blockIdx.x, I, J);
    const bool diag = I == J;
    const float *g = g_all + (int64_t)b * n_pad;
    for (int k = tid; k < SB; k += SYM_THREADS) {
        gI[k] = g[(int64_t)I * SB + k] * sc[(int64_t)I * SB + k];
        gJ[k] = g[(int64_t)J * SB + k] * sc[(int64_t)J * SB + k];
    }
    __syncthreads();
    const uint4 *blk = K + (int64_t)blockIdx.x * SB * SBC * 2;
    float col[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) col[c] = 0.f;
    float *out_rows = partial + ((int64_t)J * B + b) * n_pad + (int64_t)I * SB;
    for (int r0 = warp; r0 < SB; r0 += 8 * SYM_WARPS) {  // 8 rows per group: r0, r0 + 8, ..., r0 + 56
        float dot[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int r = r0 + 8 * k;
            const uint4 *row = blk + (int64_t)r * SBC * 2;
            uint4 hv[4], lv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                hv[u] = ld_stream_u4(row + 2 * (lane + 32 * u));
                lv[u] = ld_stream_u4(row + 2 * (lane + 32 * u) + 1);
            }
            const float gi = gI[r];
            float d = 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 g0 = *reinterpret_cast<const float4 *>(gJ + 8 * (lane + 32 * u));
                const float4 g1 = *reinterpret_cast<const float4 *>(gJ + 8 * (lane + 32 * u) + 4);
                const float gj[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
                const uint32_t hw[4] = {hv[u].x, hv[u].y, hv[u].z, hv[u].w};
                const uint32_t lw[4] = {lv[u].x, lv[u].y, lv[u].z, lv[u].w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float v0 = __uint_as_float(hw[q] << 16) + __uint_as_float(lw[q] << 16);
                    const float v1 = __uint_as_float(hw[q] & 0xffff0000u) + __uint_as_float(lw[q] & 0xffff0000u);
                    d = fmaf(v0, gj[2 * q], d);
                    d = fmaf(v1, gj[2 * q + 1], d);
                    col[8 * u + 2 * q] = fmaf(v0, gi, col[8 * u + 2 * q]);
                    col[8 * u + 2 * q + 1] = fmaf(v1, gi, col[8 * u + 2 * q + 1]);
                }
            }
            dot[k] = d;
        }
        int base = 0, cnt = 8;
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            if (cnt > 1) {
                const int h = cnt >> 1;
                const bool upper = (lane & off) != 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (k < h) {
                        const float send = upper ? dot[k] : dot[k + h];
                        const float keep = upper ? dot[k + h] : dot[k];
                        dot[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                    }
                }
                if (upper) base += h;
                cnt = h;
            } else {
                dot[0] += __shfl_xor_sync(0xffffffffu, dot[0], off);
            }
        }
        if ((lane & 3) == 0) {
            const int r = r0 + 8 * base;
            out_rows[r] = sc[(int64_t)I * SB + r] * dot[0];
        }
    }
    if (diag) return;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        float *dst = &colred[warp][8 * (lane + 32 * u)];
        *reinterpret_cast<float4 *>(dst) = make_float4(col[8 * u], col[8 * u + 1], col[8 * u + 2], col[8 * u + 3]);
        *reinterpret_cast<float4 *>(dst + 4) =
            make_float4(col[8 * u + 4], col[8 * u + 5], col[8 * u + 6], col[8 * u + 7]);
    }
    __syncthreads();
    float *out_cols = partial + ((int64_t)I * B + b) * n_pad + (int64_t)J * SB;
    for (int k = tid; k < SB; k += SYM_THREADS) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < SYM_WARPS; ++w) v += colred[w][k];
        out_cols[k] = sc[(int64_t)J * SB + k] * v;
    }
}

// ---------------------------------------------------------------- GEMM (several trajectories)
// I[b, i] = sum_j WQ[i, j] F[b, j] for B >= kGemmMinB trajectories on the FP32 plane: a
// register-tiled SIMT GEMM on the FP32 FMA pipe (the plain-FP32 counterpart of the batched
// tensor-core path), so that W is streamed once per 128 or 64 trajectories instead of once
// per trajectory.  CTA tile 128 rows (i) x GB_BN trajectories (b) x 16 columns (j) per
// step, 256 threads; thread (tm, tn) = (tid & 15, tid >> 4) owns the row pairs
// (2 tm + 32 r, 2 tm + 32 r + 1), r = 0..3, and the trajectories tn * 4 + c (plus
// 64 + tn * 4 + c when GB_BN = 128).  Accumulators are FP32 pairs along i, updated by
// fma.rn.f32x2 with the trajectory operand stored twice in shared memory (f, f): per k a
// warp reads its 32 rows' W values as one 128-byte row of pairs and its two trajectories'
// F values by broadcast.  Tiles are staged through registers into double-buffered shared
// memory (transposed: k-major).  Small node sets split K (grid z) into partial-sum slots
// that the stage kernel adds in a fixed order.
constexpr int GB_BM = 128, GB_BK = 16, GB_THREADS = 256;
constexpr int kGemmMinB = 8;

// Row strides are padded (130 floats, GB_BN + 2 pairs) so that the transposing stores of a
// warp (8 rows or trajectories x 4 k-quads) fall into distinct banks, while every row stays
// 8-byte (a) and 16-byte (b) aligned for the compute loop's vector loads.
constexpr int GB_AS = GB_BM + 2;
template <int GB_BN>
struct GemmSmem {
    float a[2][GB_BK][GB_AS];                       // W tile, k-major
    unsigned long long b[2][GB_BK][GB_BN + 2];      // (f, f) pairs, k-major
};

typedef unsigned long long u64d;
__device__ __forceinline__ u64d d_fma2(u64d a, u64d b, u64d c) {
    u64d d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64d d_pack(float lo, float hi) {
    u64d d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}

template <int GB_BN>
__global__ void __launch_bounds__(GB_THREADS, 2)
gemm_fp32_kernel(const float *__restrict__ W, const float *__restrict__ F, int64_t n_pad, int B, int64_t kchunk,
                 float *__restrict__ partial) {
    constexpr int NC = GB_BN / 16;                   // trajectories per thread (8 or 4)
    constexpr int BLD = GB_BN * 4 / GB_THREADS;      // float4 loads of the F tile per thread (2 or 1)
    extern __shared__ __align__(16) unsigned char gm_raw[];
    GemmSmem<GB_BN> &sm = *reinterpret_cast<GemmSmem<GB_BN> *>(gm_raw);
    const int tid = threadIdx.x, tm = tid & 15, tn = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * GB_BM;
    const int n0 = blockIdx.y * GB_BN;
    const int64_t k0 = (int64_t)blockIdx.z * kchunk, k1 = min(n_pad, k0 + kchunk);
    const int nkt = (int)((k1 - k0) / GB_BK);
    float4 ra[2], rb[BLD];
    auto load = [&](int kt) {
        const int64_t kb = k0 + (int64_t)kt * GB_BK;
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int idx = tid + GB_THREADS * p, r = idx >> 2, kq = idx & 3;
            ra[p] = __ldg(reinterpret_cast<const float4 *>(W + (m0 + r) * n_pad + kb + 4 * kq));
        }
#pragma unroll
        for (int p = 0; p < BLD; ++p) {
            const int idx = tid + GB_THREADS * p, c = idx >> 2, kq = idx & 3;
            const int b = n0 + c;
            rb[p] = b < B ? __ldg(reinterpret_cast<const float4 *>(F + (int64_t)b * n_pad + kb + 4 * kq))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int idx = tid + GB_THREADS * p, r = idx >> 2, kq = idx & 3;
            sm.a[buf][4 * kq + 0][r] = ra[p].x;
            sm.a[buf][4 * kq + 1][r] = ra[p].y;
            sm.a[buf][4 * kq + 2][r] = ra[p].z;
            sm.a[buf][4 * kq + 3][r] = ra[p].w;
        }
#pragma unroll
        for (int p = 0; p < BLD; ++p) {
            const int idx = tid + GB_THREADS * p, c = idx >> 2, kq = idx & 3;
            sm.b[buf][4 * kq + 0][c] = d_pack(rb[p].x, rb[p].x);
            sm.b[buf][4 * kq + 1][c] = d_pack(rb[p].y, rb[p].y);
            sm.b[buf][4 * kq + 2][c] = d_pack(rb[p].z, rb[p].z);
            sm.b[buf][4 * kq + 3][c] = d_pack(rb[p].w, rb[p].w);
        }
    };
    u64d acc[4][NC];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[r][c] = 0ull;
    if (nkt > 0) {
        load(0);
        store(0);
    }
    __syncthreads();
    for (int kt = 0; kt < nkt; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nkt) load(kt + 1);  // global loads in flight during the compute below
#pragma unroll 4
        for (int k = 0; k < GB_BK; ++k) {
            u64d bd[NC];
#pragma unroll
            for (int c2 = 0; c2 < NC; c2 += 2) {
                const int col = (c2 < 4 ? tn * 4 : 64 + tn * 4) + (c2 & 3);
                const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(&sm.b[buf][k][col]);
                bd[c2] = v.x;
                bd[c2 + 1] = v.y;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const u64d a = *reinterpret_cast<const u64d *>(&sm.a[buf][k][2 * tm + 32 * r]);
#pragma unroll
                for (int c = 0; c < NC; ++c) acc[r][c] = d_fma2(a, bd[c], acc[r][c]);
            }
        }
        if (kt + 1 < nkt) store(buf ^ 1);
        __syncthreads();
    }
    float *out = partial + (int64_t)blockIdx.z * B * n_pad;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int b = n0 + (c < 4 ? tn * 4 : 64 + tn * 4) + (c & 3);
        if (b >= B) continue;
#pragma unroll
        for (int r = 0; r < 4; ++r)
            *reinterpret_cast<u64d *>(out + (int64_t)b * n_pad + m0 + 2 * tm + 32 * r) = acc[r][c];
    }
}

// (K splits, K columns per split) of the GEMM: the split count (at most 16, each split at
// least 64 K steps) whose CTAs best fill whole waves of two CTAs per SM; each extra split
// costs one more B x n partial-sum slot, a small penalty.
static SplitPlan gemm_plan(const nf_operator *op, int B) {
    SplitPlan p{};
    const int bn = B > 64 ? 128 : 64;
    const int64_t tiles = (op->n_pad / GB_BM) * ((B + bn - 1) / bn);
    const int64_t ktiles = op->n_pad / GB_BK;
    const int64_t slots = 2 * (int64_t)num_sms();
    int s = 1;
    double best = -1.0;
    for (int c = 1; c <= 16 && (c == 1 || ktiles / c >= 64); ++c) {
        const int64_t per_c = ceil_div(ktiles, c);
        if (ceil_div(ktiles, per_c) != c) continue;
        const int64_t items = tiles * c;
        const double eff = (double)items / (double)(ceil_div(items, slots) * slots) - 0.005 * c;
        if (eff > best + 1e-9) {
            best = eff;
            s = c;
        }
    }
    const int64_t per = ceil_div(ktiles, s);
    p.rows_per_block = GB_BM;
    p.row_blocks = op->n_pad / GB_BM;
    p.splits = (int)ceil_div(ktiles, per);
    p.jchunk = per * GB_BK;
    return p;
}

static bool use_gemm(const nf_operator *op, int B) { return op->path == NF_DENSE_FP32 && B >= kGemmMinB; }

nf_status dense_init_attrs() {
    NF_CUDA_TRY(cudaFuncSetAttribute(gemm_fp32_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(GemmSmem<128>)));
    NF_CUDA_TRY(cudaFuncSetAttribute(gemm_fp32_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(GemmSmem<64>)));
    return NF_OK;
}

SplitPlan dense_plan(nf_operator *op) {
    int res = 0;
    if (op->path == NF_DENSE_FP32)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res, gemv_fp32_kernel, DG_THREADS, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res, gemv_bf16x2_kernel, DG_THREADS, 0);
    return plan_splits(op->n_pad, DG_ROWS, DG_TILE, std::max(res, 1));
}

int dense_splits(nf_operator *op, int B) {
    if (use_gemm(op, B)) return gemm_plan(op, B).splits;
    const bool sym = op->path == NF_DENSE_SYM_FP32 || op->path == NF_DENSE_SYM_BF16X2;
    return sym ? (int)(op->n_pad / SB) : dense_plan(op).splits;
}

size_t dense_sym_entries(int64_t n_pad) {
    const int64_t nb = n_pad / SB;
    return (size_t)(nb * (nb + 1) / 2) * SB * SB;
}

nf_status launch_dense_gemv(nf_operator *op, int B, cudaStream_t s, int *splits_out) {
    if (op->path == NF_DENSE_SYM_FP32 || op->path == NF_DENSE_SYM_BF16X2) {
        const int64_t nb = op->n_pad / SB;
        for (int b = 0; b < B; ++b) {
            if (op->path == NF_DENSE_SYM_FP32)
                gemv_sym_fp32_kernel<<<(unsigned)(nb * (nb + 1) / 2), SYM_THREADS, 0, s>>>(op->W32, op->g, op->n_pad,
                                                                                         B, b, op->partial);
            else
                gemv_sym_bf16x2_kernel<<<(unsigned)(nb * (nb + 1) / 2), SYM_THREADS, 0, s>>>(
                    reinterpret_cast<const uint4 *>(op->Whi), op->g, op->rs, op->n_pad, B, b, op->partial);
            NF_CUDA_TRY(cudaGetLastError());
        }
        *splits_out = (int)nb;
        return NF_OK;
    }
    if (use_gemm(op, B)) {
        const SplitPlan gp = gemm_plan(op, B);
        if (B > 64) {
            dim3 grid((unsigned)gp.row_blocks, (unsigned)((B + 127) / 128), (unsigned)gp.splits);
            gemm_fp32_kernel<128><<<grid, GB_THREADS, sizeof(GemmSmem<128>), s>>>(op->W32, op->g, op->n_pad, B,
                                                                                gp.jchunk, op->partial);
        } else {
            dim3 grid((unsigned)gp.row_blocks, (unsigned)((B + 63) / 64), (unsigned)gp.splits);
            gemm_fp32_kernel<64><<<grid, GB_THREADS, sizeof(GemmSmem<64>), s>>>(op->W32, op->g, op->n_pad, B,
                                                                              gp.jchunk, op->partial);
        }
        NF_CUDA_TRY(cudaGetLastError());
        *splits_out = gp.splits;
        return NF_OK;
    }
    const SplitPlan pl = dense_plan(op);
    dim3 grid((unsigned)pl.row_blocks, (unsigned)pl.splits);
    for (int b = 0; b < B; ++b) {
        if (op->path == NF_DENSE_FP32)
            gemv_fp32_kernel<<<grid, DG_THREADS, 0, s>>>(op->W32, op->g, op->n_pad, B, b, pl.jchunk, op->partial);
        else
            gemv_bf16x2_kernel<<<grid, DG_THREADS, 0, s>>>(op->Whi, op->Wlo, op->g, op->n_pad, B, b, pl.jchunk,
                                                           op->partial);
        NF_CUDA_TRY(cudaGetLastError());
    }
    *splits_out = pl.splits;
    return NF_OK;
}

}  // namespace nfi
