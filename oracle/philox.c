/*
 * philox.c -- Philox4x32-10 counter-based generator, written from its
 * published definition (Salmon, Moraes, Dror, Shaw, "Parallel Random
 * Numbers: As Easy as 1, 2, 3", SC'11, Sec. 4.2): ten rounds of two 32x32->64
 * multiplications with the multipliers 0xD2511F53 and 0xCD9E8D57, the key
 * bumped by the Weyl constants 0x9E3779B9 and 0xBB67AE85 between rounds.
 *
 * TEST INFRASTRUCTURE: part of the CPU oracle; it shares no code with the
 * CUDA path, which implements the same published generator on its own.
 *
 * The random numbers of the QED Monte Carlo (Sec. IV, Method I and II) are
 * drawn from this stream, so that the oracle and the GPU see the same r.
 */
#include <stdint.h>

#include "pic_oracle.h"

static void mulhilo(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void or_philox4x32_10(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out)
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo(0xD2511F53u, c[0], &hi0, &lo0);
        mulhilo(0xCD9E8D57u, c[2], &hi1, &lo1);
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* uniform deviate in (0,1) from the top 24 bits of a word: (x>>8 + 1/2) 2^-24,
 * exactly representable in both binary32 and binary64 */
double or_uniform24(uint32_t x) { return ((double)(x >> 8) + 0.5) * (1.0 / 16777216.0); }
