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
 *  - N(0,1) payloads: Box-Muller (1958) in single precision on two 24-bit
 *    uniforms in (0,1) taken from outputs 2j and 2j+1: normal 2j is
 *    r*cos(theta), normal 2j+1 is r*sin(theta), with r = sqrt(-2 ln u1) and
 *    theta = 2 pi u2 (|normal| < 5.9).
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

static inline float wl_unit24(uint64_t v)
{
    /* (k + 0.5) * 2^-24, k the top 24 bits: strictly inside (0, 1), exact. */
    return ((float)(uint32_t)(v >> 40) + 0.5f) * (1.0f / 16777216.0f);
}

/* Normals 2j and 2j+1 of the stream seeded with `seed`. */
static inline void wl_normal_pair(uint64_t seed, uint64_t j, float *z0, float *z1)
{
    float u1 = wl_unit24(wl_splitmix64_at(seed, 2 * j));
    float u2 = wl_unit24(wl_splitmix64_at(seed, 2 * j + 1));
    float r = sqrtf(-2.0f * logf(u1));
    float th = 6.28318530717958647692f * u2;
    *z0 = r * cosf(th);
    *z1 = r * sinf(th);
}

void wl_normal_f32(uint64_t seed, uint64_t first, uint64_t n, float *out)
{
    uint64_t i = 0;
    while (i < n) {
        uint64_t g = first + i;
        float z0, z1;
        wl_normal_pair(seed, g >> 1, &z0, &z1);
        if (g & 1) {
            out[i++] = z1;
        } else {
            out[i++] = z0;
            if (i < n) out[i++] = z1;
        }
    }
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
    /* Round to the OCP E4M3 grid with ties to even, saturating at +-448.
     * Normal range (|f| >= 2^-6): round the binary32 significand from 23 to 3
     * bits (add half-1 plus the kept LSB, then truncate; a carry moves into
     * the exponent), rebias 127 -> 7.  Below 2^-6 the grid step is 2^-9:
     * |f| * 2^9 is exact and nearbyintf rounds it to even (a result of 8 is
     * the code of 2^-6). */
    uint32_t b;
    memcpy(&b, &f, 4);
    uint8_t sign = (uint8_t)((b >> 24) & 0x80);
    uint32_t a = b & 0x7FFFFFFFu;
    if (a > 0x7F800000u)
        return (uint8_t)(sign | 0x7F);               /* NaN */
    if (a >= 0x43E00000u)
        return (uint8_t)(sign | 0x7E);               /* >= 448 (and inf): saturate */
    if (a < 0x3C800000u) {                           /* below 2^-6 */
        float mag;
        memcpy(&mag, &a, 4);
        return (uint8_t)(sign | (uint8_t)nearbyintf(mag * 512.0f));
    }
    uint32_t r = a + 0x7FFFFu + ((a >> 20) & 1u);
    uint32_t code = (((r >> 23) - 127u + 7u) << 3) | ((r >> 20) & 7u);
    if (code > 0x7Eu)
        code = 0x7Eu;
    return (uint8_t)(sign | code);
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
    if (dtype < 1 || dtype > 3)
        return -1;
    uint64_t i = 0;
    while (i < n) {
        uint64_t g = first + i;
        float z[2];
        wl_normal_pair(seed, g >> 1, &z[0], &z[1]);
        for (int h = (int)(g & 1); h < 2 && i < n; ++h, ++i) {
            float f = z[h];
            if (dtype == 1)
                ((float *)out)[i] = f;
            else if (dtype == 2)
                ((uint16_t *)out)[i] = wl_bf16(f);
            else
                ((uint8_t *)out)[i] = wl_fp8_e4m3(scale * f);
        }
    }
    return 0;
}

/* Pointer-chase chain: n elements, one every `stride_words` uint32 words of
 * `out` (n * stride_words words, zero elsewhere).  Element i holds the word
 * index of its successor; the successor map is a single cycle through all n
 * elements (Sattolo's algorithm, 1986), drawn with splitmix64(seed): for i
 * from n-1 down to 1, swap p[i] with p[j], j uniform in [0, i).  Returns -1 if
 * an index would not fit in 32 bits. */
int32_t wl_chase_chain(uint64_t seed, uint64_t n, uint64_t stride_words, uint32_t *out, uint32_t *perm)
{
    if (n == 0 || n * stride_words > 0xFFFFFFFFull)
        return -1;
    memset(out, 0, (size_t)(n * stride_words) * sizeof(uint32_t));
    for (uint64_t i = 0; i < n; ++i)
        perm[i] = (uint32_t)i;
    for (uint64_t i = n - 1, m = 0; i > 0; --i, ++m) {
        uint64_t j = wl_splitmix64_at(seed, m) % i; /* uniform in [0, i) */
        uint32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
    /* perm is a cyclic permutation: element i's successor is perm[i] */
    for (uint64_t i = 0; i < n; ++i)
        out[i * stride_words] = (uint32_t)(perm[i] * stride_words);
    return 0;
}
