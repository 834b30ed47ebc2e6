/* Minimum distance of the [7,4] Hamming code through the C-ABI (plain C99).
 *
 * Exit status: 0 when d = 3 was computed, 1 on a wrong result, 2 when the library
 * refused (its error message on stdout), e.g. MDIST_ECUDA on a machine without a GPU. */
#include <stdint.h>
#include <stdio.h>

#include "mdist.h"

int main(void) {
    /* G = [I_4 | P], one uint64 word per row, column i at bit i */
    const uint64_t G[4] = {
        0x01u | 0x10u | 0x20u,        /* 1000 110 */
        0x02u | 0x10u | 0x40u,        /* 0100 101 */
        0x04u | 0x20u | 0x40u,        /* 0010 011 */
        0x08u | 0x10u | 0x20u | 0x40u /* 0001 111 */
    };
    mdist_code *code = NULL;
    int rc = mdist_prepare(G, 7, 4, 1, NULL, NULL, &code);
    if (rc != MDIST_OK) {
        printf("%s\n", mdist_strerror(rc));
        return 2;
    }
    int d = 0;
    uint64_t witness[1] = {0}, message[1] = {0};
    mdist_key key;
    mdist_stats stats;
    rc = mdist_min_distance(code, &d, witness, message, &key, &stats);
    mdist_free(code);
    if (rc != MDIST_OK) {
        printf("%s\n", mdist_strerror(rc));
        return 2;
    }
    printf("d = %d, witness 0x%llx (level %d, set %d)\n", d, (unsigned long long)witness[0], key.g, key.j);
    return d == 3 ? 0 : 1;
}
