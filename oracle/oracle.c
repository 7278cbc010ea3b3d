/*
 * oracle.c -- plain, slow, obviously correct CPU oracle for the streaming
 * global-load checksum path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  It may be used only by tests/, by __graft_entry__.smoke()
 * and by bench.py's CPU-baseline / reference arm.  It shares no code, header,
 * table or constant with the CUDA path.
 *
 * What it computes (the plain definitions the GPU path must reproduce):
 *
 *  - Paper §3 "Instruments": every loaded value is folded into a sink so that
 *    no load is dead.  The folded sink here is a pair
 *        sum_u32 = (sum over all uint32 words w[i]) mod 2^32
 *        xor_u64 = XOR over j of q[j],  q[j] = w[2j] | (uint64)w[2j+1] << 32
 *    i.e. little-endian 64-bit words.  Reading the buffer P times folds every
 *    word P times (paper §3 "Allocation-size sweep": issued volume may exceed
 *    the allocation, so the buffer is re-read).
 *
 *  - Paper §3 "Fixed-work control" and §4.2 "Exact-work accounting": issued
 *    logical loads.  The library's control issues exactly bytes/16 sixteen-byte
 *    loads per pass at every K; the paper's own fixed-iteration arithmetic
 *    (iterations = floor(L / (threads*K))) and its mismatch are also given so
 *    the printed 0.024576% can be reconstructed.
 *
 *  - Paper §4.1 "Primitive baseline": a dependent pointer chase -- follow a
 *    chain of word indices a given number of steps (oracle_chase).
 *
 *  - Float payloads (precision form; no paper counterpart): the exact sum of
 *    the decoded values, computed as an FP64 Neumaier (improved Kahan-Babuska)
 *    sum in element order, plus the sum of absolute values.  Decoders follow
 *    the IEEE binary32 layout, the bfloat16 layout (upper half of binary32)
 *    and the OCP FP8 E4M3 ("fn": no infinities, S.1111.111 is NaN) layout.
 *
 * Everything is single-threaded, in index order, with no blocking.  Compiled
 * with -O2 -ffp-contract=off (no fused multiply-add, no reassociation).
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <math.h>

/* ---- integer checksum ------------------------------------------------- */

/* sum_u32 over nwords uint32 words, wrapping mod 2^32. */
uint32_t oracle_sum_u32(const uint32_t *w, uint64_t nwords)
{
    uint32_t s = 0;
    for (uint64_t i = 0; i < nwords; ++i)
        s += w[i];
    return s;
}

/* xor_u64 over nwords uint32 words taken as little-endian 64-bit pairs.
 * nwords must be even; returns 0 for nwords == 0. */
uint64_t oracle_xor_u64(const uint32_t *w, uint64_t nwords)
{
    uint64_t x = 0;
    for (uint64_t j = 0; 2 * j + 1 < nwords; ++j) {
        uint64_t q = (uint64_t)w[2 * j] | ((uint64_t)w[2 * j + 1] << 32);
        x ^= q;
    }
    return x;
}

/* The checksum of reading the buffer `passes` times: literally fold every
 * word passes times (no closed form here; the tests check the closed form). */
void oracle_checksum(const uint32_t *w, uint64_t nwords, uint64_t passes,
                     uint32_t *sum_out, uint64_t *xor_out)
{
    uint32_t s = 0;
    uint64_t x = 0;
    for (uint64_t p = 0; p < passes; ++p) {
        s += oracle_sum_u32(w, nwords);
        x ^= oracle_xor_u64(w, nwords);
    }
    *sum_out = s;
    *xor_out = x;
}

/* The checksum of the paper's fixed-iteration reads (§3 "Fixed-work
 * control", with the allocation sweep's wrap-around): nloads 16-byte loads
 * j = 0, 1, ..., nloads-1, load j reading 16-byte vector (j mod nvec) of a
 * buffer of nvec = nwords/4 vectors.  Folded literally, one load at a time.
 * nwords must be a multiple of 4; nvec == 0 gives (0, 0). */
void oracle_wrapped_checksum(const uint32_t *w, uint64_t nwords, uint64_t nloads,
                             uint32_t *sum_out, uint64_t *xor_out)
{
    uint64_t nvec = nwords / 4;
    uint32_t s = 0;
    uint64_t x = 0;
    uint64_t v = 0; /* j mod nvec */
    if (nvec == 0)
        nloads = 0;
    for (uint64_t j = 0; j < nloads; ++j) {
        const uint32_t *q = w + 4 * v;
        s += q[0] + q[1] + q[2] + q[3];
        x ^= ((uint64_t)q[0] | ((uint64_t)q[1] << 32)) ^ ((uint64_t)q[2] | ((uint64_t)q[3] << 32));
        if (++v == nvec)
            v = 0;
    }
    *sum_out = s;
    *xor_out = x;
}

/* ---- issued-load accounting ------------------------------------------- */

/* The library's fixed-work control: one 16-byte logical load per 16 bytes per
 * pass, independent of K, mechanism, CTA shape, grid and order. */
uint64_t oracle_issued_loads(uint64_t bytes, uint64_t passes)
{
    return passes * (bytes / 16);
}

/* The paper's fixed-work arithmetic (§3 Fixed-work control): iterations per
 * cell = L / (threads * K), taken as integer division, so that total issued
 * logical loads = iterations * threads * K.  Writes issued[i] for each K and
 * returns the maximum relative mismatch across the Ks, measured against the
 * largest issued count (the paper's §4.2 "exact product of iteration count and
 * per-thread offered count over the full K sweep"). */
double oracle_fixed_iteration(uint64_t target_loads, uint64_t threads,
                              const int32_t *ks, int32_t nk, uint64_t *issued)
{
    uint64_t lo = UINT64_MAX, hi = 0;
    for (int32_t i = 0; i < nk; ++i) {
        uint64_t k = (uint64_t)ks[i];
        uint64_t iters = target_loads / (threads * k);
        issued[i] = iters * threads * k;
        if (issued[i] < lo) lo = issued[i];
        if (issued[i] > hi) hi = issued[i];
    }
    if (nk == 0 || hi == 0)
        return 0.0;
    return (double)(hi - lo) / (double)hi;
}

/* ---- float decoders ---------------------------------------------------- */

enum { OR_U32 = 0, OR_F32 = 1, OR_BF16 = 2, OR_FP8_E4M3 = 3 };

static double dec_f32(uint32_t bits)
{
    float f;
    memcpy(&f, &bits, sizeof f);
    return (double)f;
}

static double dec_bf16(uint16_t h)
{
    /* bfloat16 is the upper 16 bits of an IEEE binary32. */
    return dec_f32((uint32_t)h << 16);
}

static double dec_fp8_e4m3(uint8_t b)
{
    /* OCP 8-bit floating point, E4M3: 1 sign, 4 exponent (bias 7), 3 mantissa.
     * Exponent field 0 is subnormal: value = m/8 * 2^(1-7).  The code
     * S.1111.111 is NaN; there are no infinities. */
    int s = (b >> 7) & 1;
    int e = (b >> 3) & 0xF;
    int m = b & 0x7;
    double v;
    if (e == 0xF && m == 0x7)
        return NAN;
    if (e == 0)
        v = ldexp((double)m, -9);             /* m/8 * 2^-6 */
    else
        v = ldexp((double)(8 + m), e - 7 - 3); /* (1 + m/8) * 2^(e-7) */
    return s ? -v : v;
}

/* Element size in bytes of each payload type. */
int32_t oracle_elem_bytes(int32_t dtype)
{
    switch (dtype) {
    case OR_U32: return 4;
    case OR_F32: return 4;
    case OR_BF16: return 2;
    case OR_FP8_E4M3: return 1;
    default: return 0;
    }
}

/* Decode n elements of a float payload into doubles.  Returns -1 on a bad
 * dtype. */
int32_t oracle_decode(int32_t dtype, const void *payload, uint64_t n, double *out)
{
    const uint8_t *p = (const uint8_t *)payload;
    for (uint64_t i = 0; i < n; ++i) {
        switch (dtype) {
        case OR_F32: {
            uint32_t b;
            memcpy(&b, p + 4 * i, 4);
            out[i] = dec_f32(b);
            break;
        }
        case OR_BF16: {
            uint16_t h;
            memcpy(&h, p + 2 * i, 2);
            out[i] = dec_bf16(h);
            break;
        }
        case OR_FP8_E4M3:
            out[i] = dec_fp8_e4m3(p[i]);
            break;
        default:
            return -1;
        }
    }
    return 0;
}

/* Exact-reference float sum of a payload: FP64 Neumaier summation in element
 * order (error bounded by about 2u|S| + n u^2 sum|x| with u = 2^-53), and the
 * sum of absolute values.  Returns -1 on a bad dtype. */
int32_t oracle_fsum(int32_t dtype, const void *payload, uint64_t n,
                    double *sum_out, double *abs_out)
{
    const uint8_t *p = (const uint8_t *)payload;
    double s = 0.0, c = 0.0, a = 0.0;
    if (dtype != OR_F32 && dtype != OR_BF16 && dtype != OR_FP8_E4M3)
        return -1;
    for (uint64_t i = 0; i < n; ++i) {
        double x;
        if (dtype == OR_F32) {
            uint32_t b;
            memcpy(&b, p + 4 * i, 4);
            x = dec_f32(b);
        } else if (dtype == OR_BF16) {
            uint16_t h;
            memcpy(&h, p + 2 * i, 2);
            x = dec_bf16(h);
        } else {
            x = dec_fp8_e4m3(p[i]);
        }
        double t = s + x;
        if (fabs(s) >= fabs(x))
            c += (s - t) + x;
        else
            c += (x - t) + s;
        s = t;
        a += fabs(x);
    }
    *sum_out = s + c;
    *abs_out = a;
    return 0;
}

/* ---- pointer chase ------------------------------------------------------ */

/* Paper §4.1 "Primitive baseline": a dependent pointer chain.  Starting at word
 * index `start`, replace the index by the word it points to, `steps` times, and
 * return the final index (or 0xFFFFFFFF if an index leaves the buffer). */
uint32_t oracle_chase(const uint32_t *chain, uint64_t nwords, uint32_t start, uint64_t steps)
{
    uint32_t idx = start;
    for (uint64_t s = 0; s < steps; ++s) {
        if ((uint64_t)idx >= nwords)
            return 0xFFFFFFFFu;
        idx = chain[idx];
    }
    return idx;
}
