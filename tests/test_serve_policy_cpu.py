"""The serving loop's admission policy (serve_policy.h, the code the scheduler runs),
checked on the CPU over random request sets: the admission order is by estimated seconds
minus waiting time (stable on ties); admission is first fit within the memory budget and
the slot count; and waiting lets a long job overtake fresh short ones."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2112_15083_gb300", "csrc")

CHECK = r"""
#include <stdio.h>
#include <stdint.h>
#include "serve_policy.h"

static uint64_t s = 12345;
static double rnd(void) {  /* splitmix64 -> [0, 1) */
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return (double)((z ^ (z >> 31)) >> 11) * 0x1.0p-53;
}

int main(void) {
    long bad = 0;
    for (int trial = 0; trial < 2000; trial++) {
        const int n = 1 + (int)(rnd() * 24);
        double est[32], sub[32], bytes[32];
        for (int i = 0; i < n; i++) {
            est[i] = (trial % 4 == 0) ? (double)(int)(rnd() * 4) : rnd() * 100.0;  /* ties often */
            sub[i] = (trial % 4 == 0) ? 0.0 : rnd() * 50.0;
            bytes[i] = 1e9 * (1.0 + rnd() * 60.0);
        }
        const double now = 60.0, budget = 150e9, in_use = rnd() * 100e9;
        const int n_active = (int)(rnd() * 4), max_active = 1 + (int)(rnd() * 8);
        int order[32], admit[32], seen[32] = {0};
        const int got = tn_admission(n, est, sub, bytes, now, budget, in_use, n_active, max_active, order, admit);
        /* a permutation, keys non-decreasing, ties in index order */
        for (int k = 0; k < n; k++) {
            if (order[k] < 0 || order[k] >= n || seen[order[k]]++) bad++;
            if (k > 0) {
                const double a = est[order[k - 1]] - (now - sub[order[k - 1]]);
                const double b = est[order[k]] - (now - sub[order[k]]);
                if (a > b || (a == b && order[k - 1] > order[k])) bad++;
            }
        }
        /* first fit in that order within the slots and the budget */
        double used = in_use;
        int cnt = n_active, count = 0;
        for (int k = 0; k < n; k++) {
            const int i = order[k];
            if (cnt >= max_active) { if (admit[i]) bad++; continue; }
            if (used + bytes[i] > budget) { if (admit[i]) bad++; continue; }
            if (!admit[i]) bad++;
            used += bytes[i];
            cnt++;
            count++;
        }
        if (count != got) bad++;
    }
    /* aging: a 100 s job submitted at t = 0 goes before 1 s jobs that arrive more than 99 s
       later (its key 100 - now is then below theirs, 1 - (now - t_submit)) ... */
    {
        double est[3] = {1.0, 100.0, 1.0}, sub[3] = {200.0, 0.0, 200.0}, bytes[3] = {1, 1, 1};
        int order[3], admit[3];
        tn_admission(3, est, sub, bytes, 201.0, 10.0, 0.0, 0, 1, order, admit);
        if (order[0] != 1 || !admit[1] || admit[0] || admit[2]) bad++;
    }
    /* ... and after 1 s jobs that arrive sooner (the earlier of two equal ones first) */
    {
        double est[3] = {1.0, 100.0, 1.0}, sub[3] = {50.0, 0.0, 50.0}, bytes[3] = {1, 1, 1};
        int order[3], admit[3];
        tn_admission(3, est, sub, bytes, 60.0, 10.0, 0.0, 0, 1, order, admit);
        if (order[0] != 0 || order[1] != 2 || order[2] != 1 || !admit[0] || admit[1] || admit[2]) bad++;
    }
    printf("%ld\n", bad);
    return bad != 0;
}
"""


def test_admission_policy_properties():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "a.c"), os.path.join(d, "a")
        open(src, "w").write(CHECK)
        subprocess.run([cc, "-O2", "-std=c11", "-I", CSRC, src, "-o", exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0 and r.stdout.strip() == "0", r.stdout
