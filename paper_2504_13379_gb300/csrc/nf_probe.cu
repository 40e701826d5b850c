// nf_probe.cu -- measured issue rates of the instructions the pair kernels are built from
// (no paper counterpart: the roofline of the matrix-free and adjoint kernels is a count of
// these instructions per pair divided by their rate, so the rate is measured, not assumed).
//
// One CTA of 1,024 threads per SM runs independent chains of one instruction kind; thread
// 0 reads the SM's cycle counter (clock64) at two CTA-wide barriers around the chains, so
// a CTA's rate in lane operations per clock needs no knowledge of the clock frequency.
// The entry point returns the median over the CTAs, and the wall time of the launch
// (CUDA events), from which the SM clock during the probe follows.
#include "nf_internal.cuh"

#include <algorithm>
#include <vector>

namespace nfi {

constexpr int PR_THREADS = 1024;
constexpr int PR_CHAINS = 8;   // independent dependency chains per thread
constexpr int PR_UNROLL = 8;   // chain steps per loop iteration

typedef unsigned long long u64p;

__device__ __forceinline__ u64p p_fma2(u64p a, u64p b, u64p c) {
    u64p d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64p p_pack(float lo, float hi) {
    u64p d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ float p_fma(float a, float b, float c) {
    float d;
    asm volatile("fma.rn.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float p_ex2(float a) {
    float d;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(d) : "f"(a));
    return d;
}

// kind 0: fma.rn.f32 (1 lane operation each), kind 1: fma.rn.f32x2 (2 lane operations),
// kind 2: ex2.approx.ftz.f32 (1 SFU operation), kind 3: fma.rn.f32x2 as a 4 x 2 outer
// product (8 accumulators against 4 + 2 operand registers, a different pair of operand
// registers in every instruction, as in a register-tiled GEMM; 2 lane operations each).
// cyc[blockIdx.x] = cycles of the chains.
// The FMA chains contract towards a fixed point (multiplier 0.999) and the ex2 chain maps
// [-1, 1] into itself, so every value stays finite; sink receives their sum only under a
// condition the compiler cannot rule out, so no chain is removed.
template <int KIND>
__global__ void __launch_bounds__(PR_THREADS, 1) probe_kernel(long long iters, long long *cyc, float *sink) {
    const float seed = 1e-3f * (float)(threadIdx.x & 63);
    float a[PR_CHAINS];
    u64p p[PR_CHAINS];
#pragma unroll
    for (int c = 0; c < PR_CHAINS; ++c) {
        a[c] = seed + 0.01f * c;
        p[c] = p_pack(a[c], a[c] + 0.5f);
    }
    const float m = 0.999f, k = 1e-4f;
    const u64p mp = p_pack(m, m), kp = p_pack(k, k);
    // outer-product operands (small, so the accumulators grow slowly and stay finite)
    u64p opa[PR_CHAINS / 2], opb[2];
#pragma unroll
    for (int c = 0; c < PR_CHAINS / 2; ++c) opa[c] = p_pack(1e-7f * (c + 1), 2e-7f * (c + 1) + seed * 1e-6f);
    opb[0] = p_pack(0.5f, 0.25f);
    opb[1] = p_pack(0.125f, 0.75f);
    __syncthreads();
    long long t0 = 0;
    if (threadIdx.x == 0) t0 = clock64();
    __syncthreads();
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PR_UNROLL; ++u) {
#pragma unroll
            for (int c = 0; c < PR_CHAINS; ++c) {
                if constexpr (KIND == 0) a[c] = p_fma(a[c], m, k);
                else if constexpr (KIND == 1) p[c] = p_fma2(p[c], mp, kp);
                else if constexpr (KIND == 3) p[c] = p_fma2(opa[c >> 1], opb[c & 1], p[c]);
                else a[c] = p_ex2(-a[c]) - 1.0f;  // stays in [-1, 1]: one SFU op + one add
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) cyc[blockIdx.x] = clock64() - t0;
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PR_CHAINS; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p[c]));
        s += a[c] + lo + hi;
    }
    if (s == 12345.678f) *sink = s;  // practically never true; keeps the chains live
}

}  // namespace nfi

using namespace nfi;

extern "C" nf_status nf_probe_pipe(int kind, int64_t iters, double *ops_per_clk_sm, double *sm_mhz, float *ms,
                                   void *stream) {
    clear_error();
    NF_ARG(ops_per_clk_sm && sm_mhz && ms, "outputs must be non-NULL");
    NF_ARG(kind >= 0 && kind <= 3, "kind = %d must be 0 (fma.f32), 1 (fma.f32x2), 2 (ex2) or 3 (f32x2 outer product)",
           kind);
    NF_ARG(iters >= 1 && iters <= (int64_t)1 << 24, "iters out of range");
    cudaStream_t s = as_stream(stream);
    const int grid = num_sms();
    long long *cyc = nullptr;
    float *sink = nullptr;
    NF_CUDA_TRY(cudaMallocAsync(&cyc, sizeof(long long) * grid + 64, s));
    sink = reinterpret_cast<float *>(cyc + grid);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        if (kind == 0) probe_kernel<0><<<grid, PR_THREADS, 0, s>>>(iters, cyc, sink);
        else if (kind == 1) probe_kernel<1><<<grid, PR_THREADS, 0, s>>>(iters, cyc, sink);
        else if (kind == 2) probe_kernel<2><<<grid, PR_THREADS, 0, s>>>(iters, cyc, sink);
        else probe_kernel<3><<<grid, PR_THREADS, 0, s>>>(iters, cyc, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    std::vector<long long> h(grid);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), cyc, sizeof(long long) * grid, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(cyc, s);
    if (e != cudaSuccess) return cuda_fail(e, "probe launch", __FILE__, __LINE__);
    // operations per CTA: threads x chains x unroll x iterations (x 2 lanes for f32x2)
    const double ops = (double)PR_THREADS * PR_CHAINS * PR_UNROLL * (double)iters * (kind == 1 || kind == 3 ? 2.0 : 1.0);
    std::vector<double> rate(grid);
    long long cmax = 1;
    for (int i = 0; i < grid; ++i) {
        rate[i] = ops / (double)std::max(1ll, h[i]);
        cmax = std::max(cmax, h[i]);
    }
    std::nth_element(rate.begin(), rate.begin() + grid / 2, rate.end());
    *ops_per_clk_sm = rate[grid / 2];
    *sm_mhz = (double)cmax / (*ms * 1e3);  // the slowest CTA's cycles over the launch's wall time
    return NF_OK;
}
