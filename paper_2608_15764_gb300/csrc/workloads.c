/*
 * workloads.c -- seeded synthetic inputs for the streaming-load path.
 *
 * This is the input generator only: it holds none of the checksum or
 * summation arithmetic.  Both the GPU path (via host->device copies) and the
 * CPU oracle read the bytes it writes.
 *
 *  - splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 *    generators", OOPSLA 2014; the public-domain splitmix64.c): state advances
 *    by the golden-ratio increment 0x9E3779B97F4A7C15 and each output is the
 *    (30, 27, 31) xor-shift / multiply finaliser of the state.  The counter
 *    form used here, output m of the stream seeded with s = mix(s + (m+1)*gamma),
 *    equals the sequential stream started from state s.
 *  - uint32 buffer layout: word 2m is the low half and word 2m+1 the high half
 *    of output m, so the little-endian uint64 at word 2m is output m.
 *  - N(0,1) payloads: Box-Muller (1958) on two 53-bit uniforms in (0,1):
 *    normals 2j and 2j+1 come from outputs 2j and 2j+1.
 *  - Encoders: float32 -> bfloat16 and float32 -> OCP FP8 E4M3, both round to
 *    nearest, ties to even, with E4M3 saturating to +-448.
 *
 * Compiled with -O2 -ffp-contract=off.
 */
#include <stdint.h>
#include <string.h>
#include <math.h>

#define WL_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t wl_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output m of the splitmix64 stream seeded with `seed`. */
uint64_t wl_splitmix64_at(uint64_t seed, uint64_t m)
{
    return wl_mix(seed + (m + 1) * WL_GAMMA);
}

void wl_splitmix_u64(uint64_t seed, uint64_t first, uint64_t n, uint64_t *out)
{
    for (uint64_t i = 0; i < n; ++i)
        out[i] = wl_splitmix64_at(seed, first + i);
}

/* uint32 words first_word .. first_word+nwords-1 of the buffer. */
void wl_splitmix_u32(uint64_t seed, uint64_t first_word, uint64_t nwords, uint32_t *out)
{
    for (uint64_t i = 0; i < nwords; ++i) {
        uint64_t w = first_word + i;
        uint64_t v = wl_splitmix64_at(seed, w >> 1);
        out[i] = (w & 1) ? (uint32_t)(v >> 32) : (uint32_t)v;
    }
}

static inline double wl_unit(uint64_t v)
{
    /* (k + 0.5) * 2^-53, k the top 53 bits: strictly inside (0, 1). */
    return ((double)(v >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

static inline double wl_normal_at(uint64_t seed, uint64_t i)
{
    uint64_t j = i >> 1;
    double u1 = wl_unit(wl_splitmix64_at(seed, 2 * j));
    double u2 = wl_unit(wl_splitmix64_at(seed, 2 * j + 1));
    double r = sqrt(-2.0 * log(u1));
    double th = 6.283185307179586476925286766559 * u2;
    return (i & 1) ? r * sin(th) : r * cos(th);
}

void wl_normal_f32(uint64_t seed, uint64_t first, uint64_t n, float *out)
{
    for (uint64_t i = 0; i < n; ++i)
        out[i] = (float)wl_normal_at(seed, first + i);
}

static inline uint16_t wl_bf16(float f)
{
    uint32_t b;
    memcpy(&b, &f, 4);
    if ((b & 0x7F800000u) == 0x7F800000u && (b & 0x007FFFFFu))
        return (uint16_t)((b >> 16) | 0x0040u); /* quiet NaN */
    uint32_t lsb = (b >> 16) & 1u;
    b += 0x7FFFu + lsb;
    return (uint16_t)(b >> 16);
}

void wl_f32_to_bf16(const float *in, uint64_t n, uint16_t *out)
{
    for (uint64_t i = 0; i < n; ++i)
        out[i] = wl_bf16(in[i]);
}

static inline uint8_t wl_fp8_e4m3(float f)
{
    /* Round |f| to the E4M3 grid with ties to even, saturate at 448, encode. */
    uint8_t sign = signbit(f) ? 0x80 : 0x00;
    double a = fabs((double)f);
    if (isnan(f))
        return (uint8_t)(sign | 0x7F);
    if (a >= 448.0)
        return (uint8_t)(sign | 0x7E);
    /* quantum: 2^-9 below 2^-6 (subnormals), else 2^(e-3) with 2^e <= a. */
    double q;
    if (a < 0.015625) {
        q = 0.001953125;
    } else {
        int e;
        frexp(a, &e);           /* a = f * 2^e, f in [0.5, 1) */
        q = ldexp(1.0, e - 1 - 3);
    }
    double r = nearbyint(a / q) * q; /* default rounding mode: ties to even */
    if (r > 448.0)
        r = 448.0;
    if (r == 0.0)
        return sign;
    if (r < 0.015625) {
        int m = (int)(r / 0.001953125); /* 1..7, exact */
        return (uint8_t)(sign | m);
    }
    int e;
    double fr = frexp(r, &e);        /* r = fr * 2^e, fr in [0.5, 1) */
    int m = (int)((fr * 2.0 - 1.0) * 8.0); /* exact */
    int ef = (e - 1) + 7;
    return (uint8_t)(sign | (ef << 3) | m);
}

void wl_f32_to_fp8_e4m3(const float *in, uint64_t n, float scale, uint8_t *out)
{
    for (uint64_t i = 0; i < n; ++i)
        out[i] = wl_fp8_e4m3(scale * in[i]);
}

/* Payload elements first..first+n-1 of a N(0,1) stream, encoded:
 * dtype 1 = float32, 2 = bfloat16 (RNE of the float32), 3 = FP8 E4M3 of
 * scale * float32.  Returns -1 on a bad dtype. */
int32_t wl_payload(int32_t dtype, uint64_t seed, uint64_t first, uint64_t n,
                   float scale, void *out)
{
    for (uint64_t i = 0; i < n; ++i) {
        float f = (float)wl_normal_at(seed, first + i);
        switch (dtype) {
        case 1: ((float *)out)[i] = f; break;
        case 2: ((uint16_t *)out)[i] = wl_bf16(f); break;
        case 3: ((uint8_t *)out)[i] = wl_fp8_e4m3(scale * f); break;
        default: return -1;
        }
    }
    return 0;
}
