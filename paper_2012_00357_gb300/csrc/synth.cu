// Device copy of the seeded synthetic data-set generator of dd_inputs.
//
// Not part of the DD method: it builds the material data set in place so that
// sets of 10^8 - 10^9 points need no host round trip.  Random draws come from
// the SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014) applied
// to key + (n + 1) * GAMMA; every floating-point operation is an explicitly
// rounded intrinsic (__dmul_rn, __dadd_rn, __dsqrt_rn) taken in the same order
// as the Python generator, so the two produce identical bits.
#include "dd_internal.cuh"

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t fmix64(uint64_t x) {
    x ^= x >> 30;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBull;
    x ^= x >> 31;
    return x;
}

__device__ __forceinline__ uint64_t draw(uint64_t key, uint64_t n) { return fmix64(key + (n + 1) * kGamma); }

struct SynthParams {
    double C[36];
    double lo, width, noise_std, beta;
    int law;
    uint64_t key;
};

__global__ void k_synth(SynthParams P, int64_t start, int64_t N, float *__restrict__ out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= N) return;
    const uint64_t base = (uint64_t)(start + t) * 64ull;
    double e[6], s[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        uint64_t x = draw(P.key, base + k);
        double u = __dmul_rn((double)(x >> 11), 1.1102230246251565404e-16);   // 2^-53
        e[k] = __dadd_rn(P.lo, __dmul_rn(P.width, u));
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double acc = __dmul_rn(P.C[6 * i], e[0]);
#pragma unroll
        for (int k = 1; k < 6; ++k) acc = __dadd_rn(acc, __dmul_rn(P.C[6 * i + k], e[k]));
        s[i] = acc;
    }
    if (P.law == 1) {
        double n2 = __dmul_rn(e[0], e[0]);
#pragma unroll
        for (int k = 1; k < 6; ++k) n2 = __dadd_rn(n2, __dmul_rn(e[k], e[k]));
        double fac = __dadd_rn(1.0, __dmul_rn(P.beta, __dsqrt_rn(n2)));
#pragma unroll
        for (int i = 0; i < 6; ++i) s[i] = __dmul_rn(s[i], fac);
    } else if (P.law == 2) {
        // cubic isotropic law of Eq. (9): 2 mu (E + beta E^3) + lam (tr + beta tr^3) I
        const double lam = P.C[1], mu = P.C[21];
        const double a = e[0], b = e[1], c = e[2];
        const double d = __dmul_rn(0.5, e[3]), g = __dmul_rn(0.5, e[4]), f = __dmul_rn(0.5, e[5]);
        auto dot3 = [](double x1, double y1, double x2, double y2, double x3, double y3) {
            return __dadd_rn(__dadd_rn(__dmul_rn(x1, y1), __dmul_rn(x2, y2)), __dmul_rn(x3, y3));
        };
        const double p11 = dot3(a, a, f, f, g, g), p22 = dot3(f, f, b, b, d, d);
        const double p33 = dot3(g, g, d, d, c, c), p23 = dot3(f, g, b, d, d, c);
        const double p13 = dot3(a, g, f, d, g, c), p12 = dot3(a, f, f, b, g, d);
        const double q11 = dot3(p11, a, p12, f, p13, g), q22 = dot3(p12, f, p22, b, p23, d);
        const double q33 = dot3(p13, g, p23, d, p33, c), q23 = dot3(p12, g, p22, d, p23, c);
        const double q13 = dot3(p11, g, p12, d, p13, c), q12 = dot3(p11, f, p12, b, p13, d);
        const double tr = __dadd_rn(__dadd_rn(a, b), c);
        const double h = __dmul_rn(lam, __dadd_rn(tr, __dmul_rn(P.beta, __dmul_rn(__dmul_rn(tr, tr), tr))));
        const double m2 = __dmul_rn(2.0, mu);
        s[0] = __dadd_rn(h, __dmul_rn(m2, __dadd_rn(a, __dmul_rn(P.beta, q11))));
        s[1] = __dadd_rn(h, __dmul_rn(m2, __dadd_rn(b, __dmul_rn(P.beta, q22))));
        s[2] = __dadd_rn(h, __dmul_rn(m2, __dadd_rn(c, __dmul_rn(P.beta, q33))));
        s[3] = __dmul_rn(m2, __dadd_rn(d, __dmul_rn(P.beta, q23)));
        s[4] = __dmul_rn(m2, __dadd_rn(g, __dmul_rn(P.beta, q13)));
        s[5] = __dmul_rn(m2, __dadd_rn(f, __dmul_rn(P.beta, q12)));
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        uint64_t sum = 0;
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            uint64_t x = draw(P.key, base + 8 + 6 * i + r);
            sum += (x & 0xFFFFFFFFull) + (x >> 32);
        }
        double g = __dmul_rn((double)((int64_t)sum - (int64_t)(6ull << 32)), 2.3283064365386962891e-10);  // 2^-32
        double sig = __dadd_rn(s[i], __dmul_rn(P.noise_std, g));
        out[t * 12 + i] = __double2float_rn(e[i]);
        out[t * 12 + 6 + i] = __double2float_rn(sig);
    }
}

}  // namespace

extern "C" dd_status dd_synth_dataset(dd_ctx *ctx, int law, double eps_lo, double eps_hi, double noise_std,
                                      double beta, const double *C, uint64_t seed, int64_t start, int64_t N,
                                      float *out_dev, void *stream) {
    if (!ctx) return DD_ERR_ARG;
    if (!C || !out_dev || N < 0 || start < 0 || law < 0 || law > 2)
        return dd_fail(ctx, DD_ERR_ARG, "dd_synth_dataset: bad argument");
    if (N == 0) return DD_OK;
    if (!dd_is_device_ptr(out_dev)) return dd_fail(ctx, DD_ERR_ARG, "dd_synth_dataset: out_dev must be device memory");
    SynthParams P;
    for (int i = 0; i < 36; ++i) P.C[i] = C[i];
    P.lo = eps_lo;
    P.width = eps_hi - eps_lo;
    P.noise_std = noise_std;
    P.beta = beta;
    P.law = law;
    P.key = fmix64(fmix64(seed + kGamma) + 1ull);   // stream 1: data sets
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
    DD_TRY_CUDA(ctx, cudaSetDevice(ctx->device));
    ctx->launches++;
    k_synth<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(P, start, N, out_dev);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    return DD_OK;
}

// Initial association idx_e = SplitMix64(key(seed, 3), e) mod N.
__global__ void k_init_assoc(uint64_t key, int64_t n, int64_t N, int32_t *__restrict__ idx) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) idx[e] = (int32_t)(draw(key, (uint64_t)e) % (uint64_t)N);
}

dd_status dd_init_association(dd_ctx *ctx, uint64_t seed, int64_t n, int64_t N, int32_t *idx, cudaStream_t s) {
    uint64_t key = fmix64(fmix64(seed + kGamma) + 3ull);
    ctx->launches++;
    k_init_assoc<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(key, n, N, idx);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    return DD_OK;
}
