/*
 * philox.c -- Philox4x32 with 10 rounds, restated from its published
 * definition (J. Salmon, M. Moraes, R. Dror, D. Shaw, "Parallel Random
 * Numbers: As Easy as 1, 2, 3", SC'11, Section 4.2): a 4-word counter is
 * pushed through 10 rounds of two 32x32->64 multiplies whose high halves are
 * xored with the other counter words and a 2-word key; the key is advanced by
 * the two Weyl constants between rounds.
 *
 * Test infrastructure: the CUDA path implements its own copy from the same
 * definition; the two are compared bit for bit in the GPU tests.
 */
#include "oracle.h"

/* multipliers and key increments of Philox4x32 (SC'11, Table 2 and text) */
#define PHX_M0 0xD2511F53u
#define PHX_M1 0xCD9E8D57u
#define PHX_W0 0x9E3779B9u
#define PHX_W1 0xBB67AE85u

static void phx_round(uint32_t x[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)PHX_M0 * (uint64_t)x[0];
    uint64_t p1 = (uint64_t)PHX_M1 * (uint64_t)x[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x[1] ^ k[0];
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x[3] ^ k[1];
    uint32_t y3 = lo0;
    x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3;
}

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += PHX_W0; k[1] += PHX_W1; }
        phx_round(x, k);
    }
    out[0] = x[0]; out[1] = x[1]; out[2] = x[2]; out[3] = x[3];
}

/* uniform in [0,1): the top 24 bits scaled by 2^-24, exact in FP32 and FP64 */
double or_u01(uint32_t u)
{
    return (double)(u >> 8) * (1.0 / 16777216.0);
}
