"""The byte lookup tables that the batch gathers decode through (built on the host by
gather_tables.h) reproduce the gather's bit maps: for random layouts (up to 40 layout
bits, up to 14 batch bits at random positions, up to 32 closed legs at random pattern
bits) and random elements and batch patterns, the per-byte table decode gives the stored
element that the bit-by-bit definition gives."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2112_15083_gb300", "csrc")

CHECK = r"""
#include <stdio.h>
#include "gather_tables.h"

static uint64_t s = 0x9E3779B97F4A7C15ull;
static uint64_t rnd(void) {  /* splitmix64 */
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t rest_t[5 * 256];
static uint32_t beta_t[5 * 256], sel_t[8 * 256];
static uint64_t pats[1 << 14];

int main(void) {
    long bad = 0, checked = 0;
    for (int trial = 0; trial < 400; trial++) {
        const int nbits = 1 + (int)(rnd() % 40);
        const int lb = (int)(rnd() % ((nbits < 14 ? nbits : 14) + 1));
        const int nq = (int)(rnd() % 33);
        int8_t pos_beta[16], beta_bit[16];
        int16_t q[32];
        int used[64] = {0};
        for (int t = 0; t < lb; t++) {  /* distinct positions, descending, a shuffled bit order */
            int p;
            do p = (int)(rnd() % nbits); while (used[p]);
            used[p] = 1;
        }
        for (int p = 63, t = 0; p >= 0; p--)
            if (used[p]) pos_beta[t++] = (int8_t)p;
        for (int t = 0; t < lb; t++) beta_bit[t] = (int8_t)t;
        for (int t = lb - 1; t > 0; t--) {
            const int u = (int)(rnd() % (t + 1));
            const int8_t x = beta_bit[t];
            beta_bit[t] = beta_bit[u];
            beta_bit[u] = x;
        }
        int qused[64] = {0};
        for (int i = 0; i < nq; i++) {
            int c;
            do c = (int)(rnd() % 64); while (qused[c]);
            qused[c] = 1;
            q[i] = (int16_t)c;
        }
        for (int b = 0; b < (1 << lb); b++) pats[b] = rnd();
        tn_gather_tables(nbits, lb, pos_beta, beta_bit, nq, q, rest_t, beta_t, sel_t);
        for (int k = 0; k < 2000; k++) {
            const uint64_t e = rnd() & ((1ull << nbits) - 1);
            /* definition: batch index from the batch positions, the rest in order, and the
               selector from the pattern's closed bits */
            uint64_t bidx = 0, rest = 0, sel = 0;
            int r = 0;
            for (int p = 0; p < nbits; p++) {
                int t = -1;
                for (int u = 0; u < lb; u++)
                    if (pos_beta[u] == p) t = u;
                if (t >= 0) bidx |= ((e >> p) & 1ull) << beta_bit[t];
                else rest |= ((e >> p) & 1ull) << r++;
            }
            for (int i = 0; i < nq; i++) sel |= ((pats[bidx] >> q[i]) & 1ull) << i;
            const uint64_t want = (sel << (nbits - lb)) | rest;
            /* table decode, as the device does it */
            uint64_t tr = 0;
            uint32_t tb = 0, ts = 0;
            for (int j = 0; j < 5; j++) {
                tr |= rest_t[j * 256 + ((e >> (8 * j)) & 255u)];
                tb |= beta_t[j * 256 + ((e >> (8 * j)) & 255u)];
            }
            const uint64_t pat = pats[tb];
            for (int j = 0; j < 8; j++) ts |= sel_t[j * 256 + ((pat >> (8 * j)) & 255u)];
            const uint64_t got = ((uint64_t)ts << (nbits - lb)) | tr;
            bad += got != want || tb != bidx;
            checked++;
        }
    }
    printf("%ld %ld\n", bad, checked);
    return bad != 0;
}
"""


def test_gather_tables_match_the_bit_maps():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "g.c"), os.path.join(d, "g")
        open(src, "w").write(CHECK)
        subprocess.run([cc, "-O2", "-std=c11", "-I", CSRC, src, "-o", exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        bad, checked = map(int, r.stdout.split())
        assert r.returncode == 0 and bad == 0 and checked == 400 * 2000
