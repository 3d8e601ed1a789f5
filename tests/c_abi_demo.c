/*
 * c_abi_demo.c -- the C ABI used from plain C, with no Python and no torch:
 * device buffers from the CUDA runtime, the library's calls on them.
 *
 * The graph is the one Section II-B walks through (Fig. 1): vertices 0..3,
 * edges 01 02 03 12 23, stored as a symmetric CSR with ascending rows.
 * Serial mode must give sequential greedy matching's result, mate = 1 0 3 2;
 * the parallel pass must give a maximal matching the checker accepts; the
 * same edges as a list must do the same; the pass with its result copied to
 * page-locked host memory while it runs must leave the host copy equal to
 * the device result; two copies of the graph packed as a
 * batch with local ids must give that result in each copy, replayed from a
 * CUDA graph; and the native server must return the serial result for a
 * host-memory request.
 *
 * Prints "ok" and exits 0, or prints what failed and exits 1.
 */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <cuda_runtime.h>

#include "skipper.h"

static int failed(const char *what, mm_status st)
{
    printf("%s: status %d: %s\n", what, (int)st, mm_last_error());
    return 1;
}

int main(void)
{
    const int64_t h_off[5] = {0, 3, 5, 8, 10};
    const uint32_t h_nb[10] = {1, 2, 3, 0, 2, 0, 1, 3, 0, 2};
    const uint32_t expect[4] = {1, 0, 3, 2};
    int64_t *d_off = NULL;
    uint32_t *d_nb = NULL, *d_mate = NULL, *d_src = NULL, *d_dst = NULL;
    uint32_t mate[4];
    if (cudaMalloc((void **)&d_off, sizeof h_off) != cudaSuccess ||
        cudaMalloc((void **)&d_nb, sizeof h_nb) != cudaSuccess ||
        cudaMalloc((void **)&d_mate, sizeof mate) != cudaSuccess) {
        printf("cudaMalloc failed\n");
        return 1;
    }
    cudaMemcpy(d_off, h_off, sizeof h_off, cudaMemcpyHostToDevice);
    cudaMemcpy(d_nb, h_nb, sizeof h_nb, cudaMemcpyHostToDevice);

    mm_graph *g = NULL;
    mm_status st = mm_create_csr(4, 10, d_off, d_nb, MM_CHECK_CSR, NULL, &g);
    if (st != MM_OK) return failed("mm_create_csr", st);
    mm_options o;
    mm_default_options(&o);
    o.serial = 1;
    if ((st = mm_skipper(g, &o, d_mate, NULL, 0, NULL, NULL)) != MM_OK) return failed("mm_skipper serial", st);
    cudaMemcpy(mate, d_mate, sizeof mate, cudaMemcpyDeviceToHost);
    if (memcmp(mate, expect, sizeof mate) != 0) {
        printf("serial mate %u %u %u %u, expected 1 0 3 2\n", mate[0], mate[1], mate[2], mate[3]);
        return 1;
    }
    o.serial = 0;
    if ((st = mm_skipper(g, &o, d_mate, NULL, 0, NULL, NULL)) != MM_OK) return failed("mm_skipper", st);
    mm_verdict v;
    if ((st = mm_validate(g, d_mate, NULL, 0, &v, NULL)) != MM_OK) return failed("mm_validate", st);
    if (v.flags != 0 || v.n_pairs != 2) {
        printf("parallel verdict flags %u pairs %llu\n", v.flags, (unsigned long long)v.n_pairs);
        return 1;
    }
    uint32_t *h_mate = NULL;
    if (cudaMallocHost((void **)&h_mate, sizeof mate) != cudaSuccess) {
        printf("cudaMallocHost failed\n");
        return 1;
    }
    if ((st = mm_skipper_to_host(g, &o, d_mate, h_mate, 2, NULL)) != MM_OK) return failed("mm_skipper_to_host", st);
    cudaMemcpy(mate, d_mate, sizeof mate, cudaMemcpyDeviceToHost);
    if (memcmp(mate, h_mate, sizeof mate) != 0) {
        printf("host copy %u %u %u %u differs from the device result\n", h_mate[0], h_mate[1], h_mate[2], h_mate[3]);
        return 1;
    }
    if ((st = mm_validate(g, d_mate, NULL, 0, &v, NULL)) != MM_OK || v.flags != 0 || v.n_pairs != 2)
        return failed("mm_validate after mm_skipper_to_host", st);
    if ((st = mm_skipper_to_host(g, &o, d_mate, mate, 2, NULL)) != MM_ERR_ARG)   /* pageable: refused */
        return failed("mm_skipper_to_host into pageable memory (expected MM_ERR_ARG)", st);
    cudaFreeHost(h_mate);
    mm_destroy(g);

    /* the same edges as a list (each once, one reversed) */
    const uint32_t h_src[5] = {0, 2, 0, 2, 2};
    const uint32_t h_dst[5] = {1, 0, 3, 1, 3};
    cudaMalloc((void **)&d_src, sizeof h_src);
    cudaMalloc((void **)&d_dst, sizeof h_dst);
    cudaMemcpy(d_src, h_src, sizeof h_src, cudaMemcpyHostToDevice);
    cudaMemcpy(d_dst, h_dst, sizeof h_dst, cudaMemcpyHostToDevice);
    if ((st = mm_create_coo(4, 5, d_src, d_dst, MM_CHECK_CSR, NULL, &g)) != MM_OK)
        return failed("mm_create_coo", st);
    o.serial = 1;
    if ((st = mm_skipper(g, &o, d_mate, NULL, 0, NULL, NULL)) != MM_OK) return failed("edge list serial", st);
    cudaMemcpy(mate, d_mate, sizeof mate, cudaMemcpyDeviceToHost);
    if (memcmp(mate, expect, sizeof mate) != 0) {   /* (0,1) first, then (2,3) */
        printf("edge-list serial mate %u %u %u %u\n", mate[0], mate[1], mate[2], mate[3]);
        return 1;
    }
    if ((st = mm_validate(g, d_mate, NULL, 0, &v, NULL)) != MM_OK || v.flags != 0)
        return failed("edge-list mm_validate", st);
    mm_destroy(g);

    /* two copies of the graph in one batch with local ids, from a CUDA graph */
    {
        int64_t b_off[9];
        uint32_t b_nb[20];
        const int64_t b_vb[3] = {0, 4, 8}, b_eb[3] = {0, 10, 20};
        for (int i = 0; i < 5; ++i) b_off[i] = h_off[i];
        for (int i = 1; i < 5; ++i) b_off[4 + i] = 10 + h_off[i];
        for (int i = 0; i < 20; ++i) b_nb[i] = h_nb[i % 10];   /* local ids in both copies */
        int64_t *d_boff = NULL, *d_vb = NULL, *d_eb = NULL;
        uint32_t *d_bnb = NULL, *d_bmate = NULL;
        uint64_t *d_gp = NULL, gp[2] = {0, 0};
        uint32_t bmate[8];
        cudaMalloc((void **)&d_boff, sizeof b_off);
        cudaMalloc((void **)&d_bnb, sizeof b_nb);
        cudaMalloc((void **)&d_vb, sizeof b_vb);
        cudaMalloc((void **)&d_eb, sizeof b_eb);
        cudaMalloc((void **)&d_bmate, sizeof bmate);
        cudaMalloc((void **)&d_gp, sizeof gp);
        cudaMemcpy(d_boff, b_off, sizeof b_off, cudaMemcpyHostToDevice);
        cudaMemcpy(d_bnb, b_nb, sizeof b_nb, cudaMemcpyHostToDevice);
        cudaMemcpy(d_vb, b_vb, sizeof b_vb, cudaMemcpyHostToDevice);
        cudaMemcpy(d_eb, b_eb, sizeof b_eb, cudaMemcpyHostToDevice);
        if ((st = mm_create_csr(8, 20, d_boff, d_bnb, MM_BATCH_LOCAL_IDS, NULL, &g)) != MM_OK)
            return failed("mm_create_csr (local ids)", st);
        mm_default_options(&o);
        o.serial = 1;
        o.use_graph = 1;
        for (int rep = 0; rep < 2; ++rep)
            if ((st = mm_skipper_batched(g, 2, d_vb, d_eb, &o, d_bmate, d_gp, NULL)) != MM_OK)
                return failed("mm_skipper_batched (local ids)", st);
        cudaMemcpy(bmate, d_bmate, sizeof bmate, cudaMemcpyDeviceToHost);
        cudaMemcpy(gp, d_gp, sizeof gp, cudaMemcpyDeviceToHost);
        if (memcmp(bmate, expect, sizeof expect) != 0 || memcmp(bmate + 4, expect, sizeof expect) != 0 ||
            gp[0] != 2 || gp[1] != 2) {
            printf("local-id batch mate %u %u %u %u / %u %u %u %u, pairs %llu %llu\n", bmate[0], bmate[1],
                   bmate[2], bmate[3], bmate[4], bmate[5], bmate[6], bmate[7], (unsigned long long)gp[0],
                   (unsigned long long)gp[1]);
            return 1;
        }
        o.serial = 0;
        o.warps_per_graph = 1;
        if ((st = mm_skipper_batched(g, 2, d_vb, d_eb, &o, d_bmate, NULL, NULL)) != MM_OK)
            return failed("mm_skipper_batched (local ids, parallel)", st);
        if ((st = mm_validate_batched(g, 2, d_vb, d_eb, d_bmate, &v, NULL)) != MM_OK) return failed("mm_validate_batched", st);
        if (v.flags != 0 || v.n_pairs != 4) {
            printf("local-id batch verdict flags %u pairs %llu\n", v.flags, (unsigned long long)v.n_pairs);
            return 1;
        }
        if ((st = mm_skipper(g, &o, d_bmate, NULL, 0, NULL, NULL)) != MM_ERR_UNSUPPORTED)
            return failed("mm_skipper on a local-id batch handle (expected MM_ERR_UNSUPPORTED)", st);
        mm_destroy(g);
        cudaFree(d_boff);
        cudaFree(d_bnb);
        cudaFree(d_vb);
        cudaFree(d_eb);
        cudaFree(d_bmate);
        cudaFree(d_gp);
    }

    /* one request through the native server, from host memory */
    mm_server_config c;
    mm_server_default_config(&c);
    c.opts.serial = 1;
    c.memory_bytes = 64u << 20;
    mm_server *s = NULL;
    if ((st = mm_server_create(&c, &s)) != MM_OK) return failed("mm_server_create", st);
    uint32_t out[4] = {7, 7, 7, 7};
    uint64_t ticket = 0;
    if ((st = mm_server_submit(s, 4, 10, h_off, h_nb, out, &ticket)) != MM_OK)
        return failed("mm_server_submit", st);
    mm_server_result r;
    if ((st = mm_server_wait(s, ticket, 60.0, &r)) != MM_OK) return failed("mm_server_wait", st);
    if (r.status != MM_OK || r.verdict.flags != 0 || memcmp(out, expect, sizeof out) != 0 ||
        r.done_ns < r.submit_ns) {
        printf("server: status %d flags %u mate %u %u %u %u\n", (int)r.status, r.verdict.flags,
               out[0], out[1], out[2], out[3]);
        return 1;
    }
    if ((st = mm_server_destroy(s)) != MM_OK) return failed("mm_server_destroy", st);

    cudaFree(d_off);
    cudaFree(d_nb);
    cudaFree(d_mate);
    cudaFree(d_src);
    cudaFree(d_dst);
    printf("ok\n");
    return 0;
}
