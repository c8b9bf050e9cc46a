// Device copy of the input module's counter-based generator (SplitMix64,
// Steele, Lea & Flood, OOPSLA 2014): x[J] = 2 u_J - 1 with u_J the top 53 bits
// of mix64(key + (J + 1) * GAMMA) times 2^-53, key = stream_key(seed, stream).
// Integer mixing and exact conversions only, so the values equal the host's
// (fci_inputs.vector_pm1) bit for bit; FP32 output is the rounded FP64 value.
// Holds no CI arithmetic.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kM1 = 0xBF58476D1CE4E5B9ull;
constexpr uint64_t kM2 = 0x94D049BB133111EBull;
constexpr uint64_t kStreamMul = 0xD1B54A32D192ED03ull;

__host__ __device__ inline uint64_t mix64(uint64_t z) {
    z ^= z >> 30;
    z *= kM1;
    z ^= z >> 27;
    z *= kM2;
    z ^= z >> 31;
    return z;
}

template <typename T>
__global__ void k_fill_pm1(T *x, int64_t start, int64_t n, uint64_t key) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t w = mix64(key + (uint64_t)(start + i + 1) * kGamma);
        const double u = (double)(w >> 11) * (1.0 / 9007199254740992.0);
        x[i] = (T)(2.0 * u - 1.0);
    }
}

}  // namespace

extern "C" int fci_inputs_fill_pm1(void *x, int64_t start, int64_t n, int f32, uint64_t seed, uint64_t stream,
                                   void *cuda_stream) {
    const uint64_t key = mix64(mix64(seed) ^ (stream * kStreamMul));
    const int64_t blocks = n > 0 ? ((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096) : 1;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (f32)
        k_fill_pm1<float><<<(unsigned)blocks, 256, 0, s>>>((float *)x, start, n, key);
    else
        k_fill_pm1<double><<<(unsigned)blocks, 256, 0, s>>>((double *)x, start, n, key);
    return (int)cudaGetLastError();
}
