/*
 * Philox4x64-10 counter-based generator, written for the oracle from the
 * published definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3", SC'11, Sec. 4.2: Philox-4x64 S-box, multipliers and
 * Weyl key schedule).
 *
 * TEST INFRASTRUCTURE: this file is part of the CPU oracle.  Only tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may
 * use it.  The CUDA library carries its own, separately written generator.
 *
 * The paper (Sec. 5.3) uses Mersenne Twister / MTGP32; a counter-based
 * generator replaces it so that the GPU and the oracle draw identical numbers
 * from (seed, step, substep, super-droplet id) without shared state.
 */
#include <stdint.h>

/* Round multipliers and Weyl increments of Philox-4x64 (SC'11 paper). */
#define PHX_M0 0xD2E7470EE14C6C93ULL
#define PHX_M1 0xCA5A826395121157ULL
#define PHX_W0 0x9E3779B97F4A7C15ULL /* golden ratio */
#define PHX_W1 0xBB67AE8584CAA73BULL /* sqrt(3) - 1   */

static void mul_hi_lo(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

/* One bijection: two 64x64->128 multiplies, a word permutation and key xor. */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t hi0, lo0, hi1, lo1;
        if (round > 0) { /* key schedule: bump before every round but the first */
            k0 += PHX_W0;
            k1 += PHX_W1;
        }
        mul_hi_lo(PHX_M0, c0, &hi0, &lo0);
        mul_hi_lo(PHX_M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}
