/*
 * philox.c -- oracle copy of the counter-based generator.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper names hash-based random numbers as what makes MC/DC runs
 * replicable ("Monte Carlo Neutron Transport and MC/DC"); it does not name
 * the function.  This oracle uses Philox4x32-10 as published by Salmon,
 * Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3"
 * (SC'11): ten rounds over a 4x32-bit counter and a 2x32-bit key.  Each
 * round multiplies counter words 0 and 2 by fixed odd constants, keeps the
 * high and low halves of the 64-bit products, and mixes the high halves with
 * the other two words and the round key; the key is bumped by the two Weyl
 * constants between rounds.
 */
#include <math.h>
#include "oracle.h"

#define PHILOX_M0 0xD2511F53u   /* multiplier for counter word 0 */
#define PHILOX_M1 0xCD9E8D57u   /* multiplier for counter word 2 */
#define PHILOX_W0 0x9E3779B9u   /* key bump, word 0 (golden ratio) */
#define PHILOX_W1 0xBB67AE85u   /* key bump, word 1 (sqrt(3) - 1)  */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 53 random bits (the top 53 of hi:lo) mapped to (0, 1]:
 * xi = (floor(hi:lo / 2^11) + 1) * 2^-53.  Never 0, so -log(xi) is finite. */
double orc_uniform(uint32_t hi, uint32_t lo)
{
    uint64_t bits = ((uint64_t)hi << 32) | (uint64_t)lo;
    uint64_t m = (bits >> 11) + 1u;
    return (double)m * 0x1.0p-53;
}

/* Isotropic direction: the x-cosine mu is uniform on [-1, 1] and the
 * azimuth phi uniform on [0, 2 pi) about the x axis (textbook isotropic
 * emission, Lewis & Miller). */
void orc_isotropic(double xi_mu, double xi_phi, double u[3])
{
    const double two_pi = 6.283185307179586;
    double mu = 2.0 * xi_mu - 1.0;
    double phi = two_pi * xi_phi;
    double s = sqrt(1.0 - mu * mu);
    u[0] = mu;
    u[1] = s * cos(phi);
    u[2] = s * sin(phi);
}
