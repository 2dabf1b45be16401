/* A C11 client that uses the learned picker through the C ABI alone: it
 * reads a picker checkpoint file, loads a graph from a binary file into the
 * library, picks the graph's threshold (float32 and bfloat16 inference),
 * prunes and labels at it, and writes the loaded picker back to a new file.
 *
 * Usage: picker_client CHECKPOINT GRAPH OUT_CHECKPOINT
 * GRAPH holds int64 n, int64 nnz, int64 off[n+1], int32 col[nnz] (native
 * byte order).  Prints "p32 q32 p16 q16 kept ncomp" and exits 0, or prints
 * the failed step and exits 1. */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "tectonic.h"

#define CHECK(cond)                                                   \
    do {                                                              \
        if (!(cond)) {                                                \
            char msg_[512];                                           \
            tec_last_error(msg_, sizeof msg_);                        \
            printf("failed: %s (line %d): %s\n", #cond, __LINE__, msg_); \
            return 1;                                                 \
        }                                                             \
    } while (0)

int main(int argc, char **argv) {
    FILE *f;
    int64_t n = 0, nnz = 0, *off = NULL, *dp = NULL, *dq = NULL, hp[2], hq[2], kept = -1, ncomp = -1;
    int32_t *col = NULL, *labels = NULL;
    size_t meta_len = 0;
    char *meta = NULL;
    tec_graph *g = NULL;
    tec_picker *pk = NULL;
    if (argc != 4) {
        printf("usage: picker_client CHECKPOINT GRAPH OUT_CHECKPOINT\n");
        return 1;
    }
    /* the checkpoint's meta text, kept to write it back unchanged */
    CHECK(tec_picker_file_read(argv[1], NULL, NULL, NULL, NULL, NULL, 0, &meta_len) == TEC_OK);
    meta = (char *)malloc(meta_len + 1);
    CHECK(meta != NULL);
    CHECK(tec_picker_file_read(argv[1], NULL, NULL, NULL, NULL, meta, meta_len + 1, NULL) == TEC_OK);
    f = fopen(argv[2], "rb");
    CHECK(f != NULL);
    CHECK(fread(&n, 8, 1, f) == 1 && fread(&nnz, 8, 1, f) == 1 && n > 0 && nnz >= 0);
    off = (int64_t *)malloc((size_t)(n + 1) * 8);
    col = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * 4);
    CHECK(off != NULL && col != NULL);
    CHECK(fread(off, 8, (size_t)(n + 1), f) == (size_t)(n + 1) && fread(col, 4, (size_t)nnz, f) == (size_t)nnz);
    fclose(f);
    CHECK(tec_graph_upload(off, 1, col, n, nnz, TEC_HOST_PTR | TEC_VALIDATE, NULL, &g) == TEC_OK);
    CHECK(tec_picker_load(argv[1], NULL, &pk) == TEC_OK);
    CHECK(cudaMalloc((void **)&dp, 2 * sizeof(int64_t)) == cudaSuccess);
    CHECK(cudaMalloc((void **)&dq, 2 * sizeof(int64_t)) == cudaSuccess);
    CHECK(tec_pick_threshold(g, pk, NULL, 0, 0, dp, dq) == TEC_OK);
    CHECK(tec_pick_threshold(g, pk, NULL, 0, 1, dp + 1, dq + 1) == TEC_OK);
    CHECK(tec_sync(g) == TEC_OK);
    CHECK(cudaMemcpy(hp, dp, sizeof hp, cudaMemcpyDeviceToHost) == cudaSuccess);
    CHECK(cudaMemcpy(hq, dq, sizeof hq, cudaMemcpyDeviceToHost) == cudaSuccess);
    CHECK(hp[0] >= 1 && hp[0] <= 64 && hq[0] == 128 && hp[1] >= 1 && hp[1] <= 64 && hq[1] == 128);
    CHECK(tec_prune(g, TEC_TECTONIC, hp[0], hq[0], NULL, &kept) == TEC_OK);
    CHECK(cudaMalloc((void **)&labels, (size_t)n * sizeof(int32_t)) == cudaSuccess);
    CHECK(tec_components(g, labels, &ncomp) == TEC_OK);
    CHECK(tec_picker_save(pk, argv[3], meta) == TEC_OK);
    printf("%lld %lld %lld %lld %lld %lld\n", (long long)hp[0], (long long)hq[0], (long long)hp[1], (long long)hq[1],
           (long long)kept, (long long)ncomp);
    CHECK(tec_picker_free(pk) == TEC_OK);
    CHECK(tec_graph_free(g) == TEC_OK);
    cudaFree(dp);
    cudaFree(dq);
    cudaFree(labels);
    free(off);
    free(col);
    free(meta);
    return 0;
}
