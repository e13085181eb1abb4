/* A plain C client of librasp_gb300.so: only include/rasp.h and the C
 * library, no Python. Used by tests/test_c_client.py.
 *
 *   rasp_client --no-gpu        argument checks that need no device
 *   rasp_client IN OUT          run the batch described in IN to completion
 *                               and write the final machine state to OUT
 *
 * IN (little-endian): u64 header[7] = {V, P, TW, l, s, w, flags}, then
 * u32 n[V], i64 words[P], u64 prog_off[V+1], i64 tape[TW],
 * u64 tape_off[V+1], u64 caps[V].
 * OUT: i64 i[V], i64 a[V], u64 steps[V], u8 status[V], u32 u_0[V],
 * u32 y_0[V], i64 y[V*s], i64 M[sum n]. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "rasp.h"

static int check(int rc, const char* what) {
    if (rc != RASP_OK) fprintf(stderr, "%s failed (%d): %s\n", what, rc, rasp_last_error());
    return rc;
}

static void* read_array(FILE* f, size_t count, size_t size) {
    void* p = malloc(count ? count * size : 1);
    if (p && count && fread(p, size, count, f) != count) {
        free(p);
        return NULL;
    }
    return p;
}

static int no_gpu(void) {
    const char* v = rasp_version();
    if (!v || strncmp(v, "rasp_gb300", 10) != 0) return 1;
    rasp_config cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.word_bits = 64;
    cfg.in_cap = 4;
    cfg.out_cap = 8;
    uint32_t n[3] = {64, 17, 300};
    uint64_t bytes = 0;
    if (check(rasp_batch_bytes(&cfg, 3, n, &bytes), "rasp_batch_bytes")) return 2;
    if (bytes < 8 * (64 + 18 + 300)) return 3;
    cfg.word_bits = 1;                       /* outside 2..64 */
    if (rasp_batch_bytes(&cfg, 3, n, &bytes) != RASP_EINVAL) return 4;
    if (!rasp_last_error() || !strstr(rasp_last_error(), "word_bits")) return 5;
    cfg.word_bits = 64;
    n[1] = 0;                                /* n = 0 */
    if (rasp_batch_bytes(&cfg, 3, n, &bytes) != RASP_EINVAL) return 6;
    printf("%s\n", v);
    return 0;
}

int main(int argc, char** argv) {
    if (argc == 2 && strcmp(argv[1], "--no-gpu") == 0) return no_gpu();
    if (argc != 3) {
        fprintf(stderr, "usage: %s --no-gpu | IN OUT\n", argv[0]);
        return 64;
    }
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 65;
    uint64_t h[7];
    if (fread(h, sizeof h[0], 7, f) != 7) return 66;
    const uint64_t V = h[0], P = h[1], TW = h[2];
    uint32_t* n = read_array(f, V, 4);
    int64_t* words = read_array(f, P, 8);
    uint64_t* prog_off = read_array(f, V + 1, 8);
    int64_t* tape = read_array(f, TW, 8);
    uint64_t* tape_off = read_array(f, V + 1, 8);
    uint64_t* caps = read_array(f, V, 8);
    fclose(f);
    if (!n || !words || !prog_off || !tape || !tape_off || !caps) return 67;

    rasp_config cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.in_cap = (uint32_t)h[3];
    cfg.out_cap = (uint32_t)h[4];
    cfg.word_bits = (uint32_t)h[5];
    cfg.flags = (uint32_t)h[6];
    rasp_batch* b = NULL;
    if (check(rasp_batch_create(&cfg, V, n, &b), "rasp_batch_create")) return 1;
    int rc = check(rasp_load_programs(b, words, prog_off, V, NULL), "rasp_load_programs");
    if (!rc) rc = check(rasp_load_inputs(b, tape, tape_off, caps), "rasp_load_inputs");
    if (!rc) rc = check(rasp_run(b, UINT64_MAX), "rasp_run");
    if (!rc) rc = check(rasp_sync(b), "rasp_sync");

    uint64_t total = 0;
    for (uint64_t v = 0; v < V; ++v) total += n[v];
    const uint64_t s = h[4];
    int64_t* i = malloc(8 * V);
    int64_t* a = malloc(8 * V);
    uint64_t* steps = malloc(8 * V);
    uint8_t* status = malloc(V);
    uint32_t* uhead = malloc(4 * V);
    uint32_t* ylen = malloc(4 * V);
    int64_t* y = malloc(s ? 8 * V * s : 1);
    int64_t* mem = malloc(8 * total);
    if (!i || !a || !steps || !status || !uhead || !ylen || !y || !mem) rc = RASP_ENOMEM;
    if (!rc) {
        rasp_state_view view = {i, a, steps, status, uhead, ylen, s ? y : NULL, mem, total};
        rc = check(rasp_read_state(b, 0, V, &view), "rasp_read_state");
    }
    rasp_batch_destroy(b);
    if (rc) return 2;
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 68;
    int ok = fwrite(i, 8, V, o) == V && fwrite(a, 8, V, o) == V && fwrite(steps, 8, V, o) == V &&
             fwrite(status, 1, V, o) == V && fwrite(uhead, 4, V, o) == V && fwrite(ylen, 4, V, o) == V &&
             fwrite(y, 8, V * s, o) == V * s && fwrite(mem, 8, total, o) == total;
    fclose(o);
    return ok ? 0 : 69;
}
