// internal.cuh -- definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/paam_rta.h"

#define PAAM_CUDA_TRY(expr)                                    \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) {                               \
            paam_note_cuda_error(e_, #expr, __FILE__, __LINE__); \
            return PAAM_E_CUDA;                                \
        }                                                      \
    } while (0)

void paam_note_cuda_error(cudaError_t e, const char *expr, const char *file, int line);

struct paam_ctx {
    int device;
    int n_sm;
    int max_smem_optin;
    int32_t *d_err; // device error word used by validation (first error wins)
};

// Device copy of a validated batch: the same SoA/CSR arrays as
// paam_systems_view, all inside one allocation.
struct paam_batch {
    paam_ctx *ctx;
    int64_t n_sys, n_chain, n_cb, n_seg, n_exec;
    int64_t *sys_chain_off, *chain_cb_off, *cb_seg_off, *T, *D, *E, *A, *sys_exec_off;
    int32_t *prio, *exec, *exec_core, *exec_prio; // exec_prio NULL => derived
    uint8_t *spin;
    int32_t max_chains; // largest chain count of any system
    int32_t max_exec;
    void *block;
    size_t block_bytes;
};

// Read-only view handed to the kernels.
struct BatchDev {
    int64_t n_sys;
    const int64_t *__restrict__ sys_chain_off;
    const int64_t *__restrict__ chain_cb_off;
    const int64_t *__restrict__ cb_seg_off;
    const int64_t *__restrict__ T;
    const int64_t *__restrict__ D;
    const int64_t *__restrict__ E;
    const int64_t *__restrict__ A;
    const int64_t *__restrict__ sys_exec_off;
    const int32_t *__restrict__ prio;
    const int32_t *__restrict__ exec;
    const int32_t *__restrict__ exec_core;
    const int32_t *__restrict__ exec_prio;
    const uint8_t *__restrict__ spin;
};

struct AnalysisParams {
    int32_t n_buckets;
    int32_t pad_;
    int64_t eps;
    int64_t kappa;
};

inline BatchDev batch_dev(const paam_batch *b)
{
    BatchDev d;
    d.n_sys = b->n_sys;
    d.sys_chain_off = b->sys_chain_off;
    d.chain_cb_off = b->chain_cb_off;
    d.cb_seg_off = b->cb_seg_off;
    d.T = b->T;
    d.D = b->D;
    d.E = b->E;
    d.A = b->A;
    d.sys_exec_off = b->sys_exec_off;
    d.prio = b->prio;
    d.exec = b->exec;
    d.exec_core = b->exec_core;
    d.exec_prio = b->exec_prio;
    d.spin = b->spin;
    return d;
}

// Analysis launcher (analyze.cu).
int paam_launch_analysis(const paam_batch *b, const AnalysisParams &p, int64_t *R, uint8_t *status,
                         uint8_t *verdict, cudaStream_t stream);
