// Byte lookup tables of a batch gather's bit maps, built on the host (C-compatible; a CPU
// test checks them against the maps' bit-by-bit definition).
//
// A gathered operand's element e has nbits layout bits; batch bit beta_bit[t] sits at
// position pos_beta[t] (t < lb) and the other bits, in ascending order, are the stored
// element's low bits ("rest").  It reads the stored element (sel << (nbits - lb)) | rest,
// where sel packs bits q[0], q[1], ... (i < nq) of the batch's pattern.  The device decode
// ORs one entry per byte: for byte j of e and value x, rest[j*256 + x] and beta[j*256 + x]
// are the contributions of x << 8j to rest and to the batch index (j < 5, so nbits <= 40);
// sel[j*256 + x] is that of byte j of the 64-bit pattern (j < 8).
#pragma once

#include <stdint.h>

static inline void tn_gather_tables(int nbits, int lb, const int8_t *pos_beta, const int8_t *beta_bit, int nq,
                                    const int16_t *q, uint64_t *rest, uint32_t *beta, uint32_t *sel) {
    int bt[64], rank[64];
    for (int p = 0; p < 64; p++) bt[p] = -1;
    for (int t = 0; t < lb; t++) bt[pos_beta[t]] = beta_bit[t];
    for (int p = 0, r = 0; p < 64; p++) rank[p] = bt[p] >= 0 ? -1 : r++;
    for (int i = 0; i < 5 * 256; i++) {
        rest[i] = 0;
        beta[i] = 0;
    }
    for (int i = 0; i < 8 * 256; i++) sel[i] = 0;
    for (int j = 0; j < 5; j++)
        for (int x = 0; x < 256; x++)
            for (int b = 0; b < 8; b++) {
                const int p = 8 * j + b;
                if (!((x >> b) & 1) || p >= nbits) continue;
                if (bt[p] >= 0) beta[j * 256 + x] |= 1u << bt[p];
                else rest[j * 256 + x] |= 1ull << rank[p];
            }
    for (int j = 0; j < 8; j++)
        for (int x = 0; x < 256; x++)
            for (int i = 0; i < nq; i++) {
                const int c = q[i] - 8 * j;
                if (c >= 0 && c < 8 && ((x >> c) & 1)) sel[j * 256 + x] |= 1u << i;
            }
}
