/* Generated by oracle/gen_gauss_cdt.py -- do not edit.
 * Inversion table of the discrete Gaussian (sigma = 3.2, |e| <= 19):
 * T_j = floor(2^64 * P(e <= -19 + j)), j = 0..37. */
#ifndef HE_ORACLE_GAUSS_CDT_H
#define HE_ORACLE_GAUSS_CDT_H
#define OR_GAUSS_BOUND 19u
static const unsigned long long OR_GAUSS_CDT[2 * OR_GAUSS_BOUND] = {
    0x0000000bd798c7acull, /* e <= -19 */
    0x00000053f5e234f7ull, /* e <= -18 */
    0x000001e24b89625aull, /* e <= -17 */
    0x000009adbc7900e1ull, /* e <= -16 */
    0x00002d17ca1e3a82ull, /* e <= -15 */
    0x0000bf05ff772ee2ull, /* e <= -14 */
    0x0002e06843bbf95dull, /* e <= -13 */
    0x000a19062dceb033ull, /* e <= -12 */
    0x00204c0ded173b17ull, /* e <= -11 */
    0x005e3163ffc656a8ull, /* e <= -10 */
    0x00fab6a7e614dfaeull, /* e <= -9 */
    0x0261b16e99bc14f8ull, /* e <= -8 */
    0x054c69348bbc9867ull, /* e <= -7 */
    0x0acd276539458231ull, /* e <= -6 */
    0x143796b3c337f00bull, /* e <= -5 */
    0x22d43df09de40e7aull, /* e <= -4 */
    0x37651d96aa4fb429ull, /* e <= -3 */
    0x51a5da2b40f1bff1ull, /* e <= -2 */
    0x700ad4bf5a6e80e2ull, /* e <= -1 */
    0x8ff52b40a5917f1dull, /* e <= 0 */
    0xae5a25d4bf0e400eull, /* e <= 1 */
    0xc89ae26955b04bd6ull, /* e <= 2 */
    0xdd2bc20f621bf185ull, /* e <= 3 */
    0xebc8694c3cc80ff4ull, /* e <= 4 */
    0xf532d89ac6ba7dceull, /* e <= 5 */
    0xfab396cb74436798ull, /* e <= 6 */
    0xfd9e4e916643eb07ull, /* e <= 7 */
    0xff05495819eb2051ull, /* e <= 8 */
    0xffa1ce9c0039a957ull, /* e <= 9 */
    0xffdfb3f212e8c4e8ull, /* e <= 10 */
    0xfff5e6f9d2314fccull, /* e <= 11 */
    0xfffd1f97bc4406a2ull, /* e <= 12 */
    0xffff40fa0088d11dull, /* e <= 13 */
    0xffffd2e835e1c57dull, /* e <= 14 */
    0xfffff6524386ff1eull, /* e <= 15 */
    0xfffffe1db4769da5ull, /* e <= 16 */
    0xffffffac0a1dcb08ull, /* e <= 17 */
    0xfffffff428673853ull, /* e <= 18 */
};
#endif
