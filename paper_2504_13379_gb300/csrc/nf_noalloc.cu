// nf_noalloc.cu -- an allocation-free variant of the matrix-free nonlocal sum.
//
// Some callers cannot allocate device memory at the moment they need the sum: code
// that runs while another component owns every allocation (a host framework that
// forbids allocation inside its operator callbacks, a fixed-budget embedded or
// real-time loop), or code paths where a cudaMalloc would synchronise the device at a
// bad time.  nf_nonlocal_apply_noalloc serves them: it needs no operator handle and
// allocates nothing.  Its working memory -- the packed node tile array, the firing
// rates and the per-split partial sums -- lives in one file-scope device array of
// fixed size, which every GPU that loads this library keeps until the process exits.
//
// The array is shared by every call: each call rewrites the parts it reads (node
// and firing-rate arrays including their zero padding) before using them, so no call
// depends on an earlier call's contents, but calls whose work overlaps on the GPU
// (for example on two streams at once) race on the array and must be serialised by
// the caller.
#include "nf_internal.cuh"

#include <mutex>

namespace nfi {

constexpr int64_t kNoallocMaxN = 32768;   // largest n accepted (n_pad <= 32768)
constexpr int kNoallocMaxSplits = 16;     // column splits of the pair kernel

// layout: [x4: kNoallocMaxN float4][g: kNoallocMaxN float][partial: splits x kNoallocMaxN float][flag]
constexpr size_t kOffX4 = 0;
constexpr size_t kOffG = kOffX4 + sizeof(float4) * kNoallocMaxN;
constexpr size_t kOffPartial = kOffG + sizeof(float) * kNoallocMaxN;
constexpr size_t kOffFlag = kOffPartial + sizeof(float) * kNoallocMaxSplits * kNoallocMaxN;
constexpr size_t kScratchBytes = kOffFlag + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array, looked up once per device with that device
// current (in host code the array's name is only a host-side stand-in).
static unsigned char *scratch_address(nf_status *st) {
    static std::mutex mu;
    static unsigned char *addr[64] = {nullptr};
    const int d = device_id();
    if (d < 0 || d >= 64) {
        *st = fail(NF_ERR_UNSUPPORTED, "device ordinal %d out of range", d);
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[d]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            *st = cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
            return nullptr;
        }
        addr[d] = static_cast<unsigned char *>(p);
    }
    *st = NF_OK;
    return addr[d];
}

// x4[j] = (x, y, z, 0), g[j] = q_j f(u_j) for j < n; zeros in the padding; flag = 0.
__global__ void noalloc_pack_kernel(const float *__restrict__ x, const float *__restrict__ q,
                                    const float *__restrict__ u, int64_t n, int64_t n_pad, float beta, float theta,
                                    float4 *__restrict__ x4, float *__restrict__ g, int *__restrict__ flag) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) *flag = 0;
    if (j >= n_pad) return;
    if (j < n) {
        x4[j] = make_float4(x[3 * j], x[3 * j + 1], x[3 * j + 2], 0.f);
        g[j] = q[j] * (1.0f / (1.0f + expf(-beta * (u[j] - theta))));
    } else {
        x4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        g[j] = 0.f;
    }
}

__global__ void noalloc_reduce_kernel(const float *__restrict__ partial, int splits, int64_t n, int64_t n_pad,
                                      float *__restrict__ I) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float acc = 0.f;
    for (int sp = 0; sp < splits; ++sp) acc += partial[(int64_t)sp * n_pad + i];
    I[i] = acc;
}

}  // namespace nfi

using namespace nfi;

extern "C" nf_status nf_nonlocal_apply_noalloc(const float *x, const float *q, int64_t n, nf_kernel kp,
                                               const float *u, float beta, float theta, float *I, void *stream) {
    clear_error();
    NF_ARG(x && q && u && I, "x, q, u and I must be non-NULL device pointers");
    NF_ARG(n >= 1 && n <= kNoallocMaxN, "n = %lld outside 1..%lld (the fixed scratch size of this entry point)",
           (long long)n, (long long)kNoallocMaxN);
    NF_ARG(kp.s1 > 0.f && kp.s2 > 0.f, "s1, s2 must be > 0");
    NF_ARG(std::isfinite(kp.period) && kp.period >= 0.f, "period must be finite and >= 0");
    nf_status st = NF_OK;
    unsigned char *base = scratch_address(&st);
    if (!base) return st;
    NF_TRY(mf_init_attrs());
    cudaStream_t s = as_stream(stream);
    const int64_t n_pad = round_up(n, kNodePad);
    float4 *x4 = reinterpret_cast<float4 *>(base + kOffX4);
    float *g = reinterpret_cast<float *>(base + kOffG);
    float *partial = reinterpret_cast<float *>(base + kOffPartial);
    int *flag = reinterpret_cast<int *>(base + kOffFlag);
    noalloc_pack_kernel<<<(unsigned)ceil_div(n_pad, 256), 256, 0, s>>>(x, q, u, n, n_pad, beta, theta, x4, g, flag);
    NF_CUDA_TRY(cudaGetLastError());
    int splits = 1;
    NF_TRY(launch_mf_pair_single(x4, g, n_pad, kp, kNoallocMaxSplits, partial, flag, s, &splits));
    noalloc_reduce_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(partial, splits, n, n_pad, I);
    NF_CUDA_TRY(cudaGetLastError());
    return NF_OK;
}
