/* A plain C consumer of include/spfhe.h: plans an Alg. 1 merge and asks the
 * rotation-base tuner for a base, through the C ABI only (host-side entry
 * points; no GPU needed).  Prints one line per result. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "spfhe.h"

int main(void)
{
    /* A (3 x 4, CSR) and B (4 x 2, CSC) */
    const int32_t a_ptr[] = {0, 2, 2, 4}, a_idx[] = {0, 3, 1, 3};
    const int32_t b_ptr[] = {0, 2, 3}, b_idx[] = {0, 3, 1};
    spfhe_sparse_meta A = {3, 4, 4, a_ptr, a_idx};
    spfhe_sparse_meta B = {4, 2, 3, b_ptr, b_idx};
    uint64_t n = 0;
    if (spfhe_plan_matches(&A, &B, NULL, &n) != SPFHE_OK) return 1;
    int32_t *m = malloc(5 * (size_t)n * sizeof(int32_t));
    if (!m || spfhe_plan_matches(&A, &B, m, &n) != SPFHE_OK) return 2;
    for (uint64_t r = 0; r < n; ++r)
        printf("match %d %d %d %d %d\n", m[5 * r], m[5 * r + 1], m[5 * r + 2], m[5 * r + 3], m[5 * r + 4]);
    free(m);
    uint32_t base = 0;
    uint64_t ks = 0, bytes = 0;
    if (spfhe_tune_rotation_base(6, 4, 2, 2, &A, &B, (uint64_t)1 << 30, &base, &ks, &bytes) != SPFHE_OK) return 3;
    printf("base %u ks %llu bytes %llu\n", base, (unsigned long long)ks, (unsigned long long)bytes);
    /* a malformed CSR (index out of range) is refused with a message */
    const int32_t bad_idx[] = {0, 9, 1, 3};
    spfhe_sparse_meta bad = {3, 4, 4, a_ptr, bad_idx};
    const spfhe_status st = spfhe_plan_matches(&bad, &B, NULL, &n);
    printf("bad %d %s\n", (int)st, spfhe_last_error());
    printf("classes %d %s\n", spfhe_prof_classes(), spfhe_prof_class_name(0));
    return 0;
}
