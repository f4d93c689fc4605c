// mpm_selfcheck.cu -- mpm_check_fixed_rounding: the 32-bit rounding path of
// the fixed-point quantiser against the 64-bit conversion, on every binary32
// input it is used for.
//
// Compiled into the same translation unit as mpm_api.cu (included at its end).

namespace mpm {

constexpr int kCheckThreads = 256;

__global__ void __launch_bounds__(kCheckThreads) k_check_f2ll(unsigned long long* bad, uint32_t* first)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long n = 0;
    uint32_t f = 0xffffffffu;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (1ull << 32); i += stride) {
        const float v = __uint_as_float((uint32_t)i);
        // every input the P2G bound admits to the 32-bit path: |v| < 2^31
        if (!(fabsf(v) < 2147483648.f)) continue;
        if (round_ll<true>(v) != round_ll<false>(v)) {
            ++n;
            if ((uint32_t)i < f) f = (uint32_t)i;
        }
    }
    if (n) {
        atomicAdd(bad, n);
        atomicMin(first, f);
    }
}

}  // namespace mpm

extern "C" mpm_status mpm_check_fixed_rounding(uint64_t* mismatches, uint32_t* first)
{
    using namespace mpm;
    if (!mismatches || !first) return fail(nullptr, MPM_EINVAL, "mpm_check_fixed_rounding: NULL pointer");
    struct Out {
        unsigned long long bad;
        uint32_t first;
    };
    Out* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(Out));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, MPM_ENOMEM, "mpm_check_fixed_rounding: cudaMalloc failed");
    }
    Out h = {0ull, 0xffffffffu};
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess || sms < 1) {
        cudaGetLastError();
        sms = 148;
    }
    e = cudaMemcpy(d, &h, sizeof h, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_check_f2ll<<<sms * 8, kCheckThreads>>>(&d->bad, &d->first);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, MPM_ECUDA, std::string("mpm_check_fixed_rounding: ") + cudaGetErrorString(e));
    }
    *mismatches = h.bad;
    *first = h.first;
    return MPM_OK;
}
