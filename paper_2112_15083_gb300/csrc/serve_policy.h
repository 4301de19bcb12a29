// Admission policy of the serving loop (C-compatible host code; a CPU test checks its
// properties).  Planned requests are ordered by estimated GPU seconds minus the time they
// have waited (shortest job first, aged so that long jobs are not starved; a stable order),
// then admitted first-fit: a request is admitted while fewer than max_active requests are
// active and its device-memory estimate fits the budget beside the requests already
// admitted; one that does not fit is skipped and the next one tried.
#pragma once

// est_s, t_submit, bytes: the n planned requests.  order receives their indices in the
// admission order; admit[i] is set to 1 for admitted request i (0 otherwise).  Returns
// the number admitted.
static inline int tn_admission(int n, const double *est_s, const double *t_submit, const double *bytes, double now,
                               double budget, double bytes_in_use, int n_active, int max_active, int *order,
                               int *admit) {
    for (int i = 0; i < n; i++) {
        order[i] = i;
        admit[i] = 0;
    }
    // stable insertion sort by est_s - (now - t_submit)
    for (int i = 1; i < n; i++) {
        const int x = order[i];
        const double kx = est_s[x] - (now - t_submit[x]);
        int j = i - 1;
        while (j >= 0 && est_s[order[j]] - (now - t_submit[order[j]]) > kx) {
            order[j + 1] = order[j];
            j--;
        }
        order[j + 1] = x;
    }
    int admitted = 0;
    for (int k = 0; k < n; k++) {
        const int i = order[k];
        if (n_active + admitted >= max_active) break;
        if (bytes_in_use + bytes[i] > budget) continue;
        bytes_in_use += bytes[i];
        admit[i] = 1;
        admitted++;
    }
    return admitted;
}
