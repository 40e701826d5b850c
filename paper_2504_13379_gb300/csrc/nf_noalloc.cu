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
// and firing-rate arrays including their zero padding, the error flag) before using
// them, so no call depends on an earlier call's contents, but calls whose work overlaps
// on the GPU (for example on two streams at once) race on the array and must be
// serialised by the caller.
//
// Failure reporting without a host round trip: the pair kernel records a bounded wait
// that gave up in the array's flag word (and then skips its partial sums); the final
// reduction reads the flag and, if it is set, writes NaN to every output entry instead
// of adding partial sums that were never written.  nf_noalloc_status reads the flag back.
//
// The array's device address is looked up once per device and cached; the cache assumes
// the device's primary context lives until the process exits (after cudaDeviceReset the
// cached address would be stale).
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

// I[i] = sum of the splits' partial sums, in split order; NaN everywhere if a pair kernel
// block gave up waiting (its partial sums were not written).
__global__ void noalloc_reduce_kernel(const float *__restrict__ partial, int splits, int64_t n, int64_t n_pad,
                                      const int *__restrict__ flag, float *__restrict__ I) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (*flag != 0) {
        I[i] = __int_as_float(0x7fc00000);
        return;
    }
    const float acc = sum_slots(partial + i, n_pad, splits);
    I[i] = acc;
}

// Stand-in for a pair kernel that gave up waiting: records a timeout in the flag.
__global__ void noalloc_set_flag_kernel(int *flag, int code) { *flag = code; }

// Column splits of a call on n_pad padded nodes (the partial-sum rows it writes).
static int noalloc_splits(int64_t n_pad) { return plan_mf_pair_single(n_pad, kNoallocMaxSplits).splits; }

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
    noalloc_reduce_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(partial, splits, n, n_pad, flag, I);
    NF_CUDA_TRY(cudaGetLastError());
    return NF_OK;
}

extern "C" nf_status nf_noalloc_status(void *stream) {
    clear_error();
    nf_status st = NF_OK;
    unsigned char *base = scratch_address(&st);
    if (!base) return st;
    cudaStream_t s = as_stream(stream);
    NF_CUDA_TRY(cudaStreamSynchronize(s));
    int flag = 0;
    NF_CUDA_TRY(cudaMemcpy(&flag, base + kOffFlag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag == DEV_TIMEOUT) return fail(NF_ERR_TIMEOUT, "a bounded wait of the last allocation-free call gave up");
    if (flag != 0) return fail(NF_ERR_CUDA, "device error flag %d", flag);
    return NF_OK;
}

extern "C" nf_status nf_noalloc_limits(int64_t n, int64_t *max_n, int *max_splits, int *splits) {
    clear_error();
    NF_ARG(max_n && max_splits && splits, "outputs must be non-NULL");
    NF_ARG(n >= 1 && n <= kNoallocMaxN, "n = %lld outside 1..%lld", (long long)n, (long long)kNoallocMaxN);
    NF_TRY(mf_init_attrs());
    *max_n = kNoallocMaxN;
    *max_splits = kNoallocMaxSplits;
    *splits = noalloc_splits(round_up(n, kNodePad));
    return NF_OK;
}

extern "C" nf_status nf_selftest_noalloc_flag(int64_t n, float *I, void *stream) {
    clear_error();
    NF_ARG(I, "I must be a non-NULL device pointer");
    NF_ARG(n >= 1 && n <= kNoallocMaxN, "n = %lld outside 1..%lld", (long long)n, (long long)kNoallocMaxN);
    nf_status st = NF_OK;
    unsigned char *base = scratch_address(&st);
    if (!base) return st;
    cudaStream_t s = as_stream(stream);
    int *flag = reinterpret_cast<int *>(base + kOffFlag);
    float *partial = reinterpret_cast<float *>(base + kOffPartial);
    noalloc_set_flag_kernel<<<1, 1, 0, s>>>(flag, DEV_TIMEOUT);
    NF_CUDA_TRY(cudaGetLastError());
    noalloc_reduce_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(partial, 1, n, round_up(n, kNodePad), flag, I);
    NF_CUDA_TRY(cudaGetLastError());
    return NF_OK;
}
