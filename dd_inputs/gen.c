/* C copy of the seeded data-set generator of dd_inputs/__init__.py (same
 * SplitMix64 counter stream, same operation order, no fused multiply-add:
 * compile with -ffp-contract=off).  Input generation only; no step of the DD
 * method.  Used where a data set of 10^8 - 10^9 points has to be produced on
 * the host chunk by chunk. */
#include <math.h>
#include <stdint.h>

#define DDI_GAMMA 0x9E3779B97F4A7C15ull

static uint64_t ddi_fmix64(uint64_t x)
{
    x ^= x >> 30;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBull;
    x ^= x >> 31;
    return x;
}

static uint64_t ddi_draw(uint64_t key, uint64_t n) { return ddi_fmix64(key + (n + 1) * DDI_GAMMA); }

uint64_t ddi_stream_key(uint64_t seed, uint64_t stream)
{
    return ddi_fmix64(ddi_fmix64(seed + DDI_GAMMA) + stream);
}

/* Points start .. start+n-1 into out [n x 12] (float32): law 0 linear,
 * law 1 nonlinear (sigma = C eps (1 + beta |eps|)), law 2 the cubic law of
 * Eq. (9) with the Lame constants of C, Irwin-Hall noise. */
void ddi_make_dataset(int law, double lo, double hi, double noise_std, double beta, const double *C,
                      uint64_t seed, int64_t start, int64_t n, float *out)
{
    const uint64_t key = ddi_stream_key(seed, 1);
    const double width = hi - lo;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < n; ++t) {
        const uint64_t base = (uint64_t)(start + t) * 64ull;
        double e[6], s[6];
        for (int k = 0; k < 6; ++k) {
            double u = (double)(ddi_draw(key, base + k) >> 11) * 1.1102230246251565404e-16;
            e[k] = lo + width * u;
        }
        for (int i = 0; i < 6; ++i) {
            double acc = C[6 * i] * e[0];
            for (int k = 1; k < 6; ++k) acc = acc + C[6 * i + k] * e[k];
            s[i] = acc;
        }
        if (law == 1) {
            double n2 = e[0] * e[0];
            for (int k = 1; k < 6; ++k) n2 = n2 + e[k] * e[k];
            double fac = 1.0 + beta * sqrt(n2);
            for (int i = 0; i < 6; ++i) s[i] = s[i] * fac;
        } else if (law == 2) {
            /* cubic isotropic law of Eq. (9) with the Lame constants of C */
            const double lam = C[1], mu = C[21];
            const double a = e[0], b = e[1], c = e[2], d = 0.5 * e[3], g = 0.5 * e[4], f = 0.5 * e[5];
            const double p11 = (a * a + f * f) + g * g, p22 = (f * f + b * b) + d * d;
            const double p33 = (g * g + d * d) + c * c, p23 = (f * g + b * d) + d * c;
            const double p13 = (a * g + f * d) + g * c, p12 = (a * f + f * b) + g * d;
            const double q11 = (p11 * a + p12 * f) + p13 * g, q22 = (p12 * f + p22 * b) + p23 * d;
            const double q33 = (p13 * g + p23 * d) + p33 * c, q23 = (p12 * g + p22 * d) + p23 * c;
            const double q13 = (p11 * g + p12 * d) + p13 * c, q12 = (p11 * f + p12 * b) + p13 * d;
            const double tr = (a + b) + c;
            const double h = lam * (tr + beta * ((tr * tr) * tr));
            const double m2 = 2.0 * mu;
            s[0] = h + m2 * (a + beta * q11);
            s[1] = h + m2 * (b + beta * q22);
            s[2] = h + m2 * (c + beta * q33);
            s[3] = m2 * (d + beta * q23);
            s[4] = m2 * (g + beta * q13);
            s[5] = m2 * (f + beta * q12);
        }
        for (int i = 0; i < 6; ++i) {
            uint64_t sum = 0;
            for (int r = 0; r < 6; ++r) {
                uint64_t x = ddi_draw(key, base + 8 + 6 * i + r);
                sum += (x & 0xFFFFFFFFull) + (x >> 32);
            }
            double g = (double)((int64_t)sum - (int64_t)(6ull << 32)) * 2.3283064365386962891e-10;
            out[t * 12 + i] = (float)e[i];
            out[t * 12 + 6 + i] = (float)(s[i] + noise_std * g);
        }
    }
}
