// handles.h -- host-side definitions of the libifem handles (internal;
// shared by the translation units that implement entry points).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/ifem.h"
#include "common.cuh"

using namespace ifem;

struct ifem_ctx_s {
    ifem_config cfg;
    int n_sm = 0;
    int tile = 8;
    std::string err;
    unsigned long long *d_status = nullptr;
    unsigned long long *h_status = nullptr;
    cudaEvent_t ev[6] = {};
    int ev_ok = 0;
    int ev_recorded = 0;
    int ev_fused = 0;   // the recorded step fused interpolation into the spread
    int acc64 = 0;
    int staged = 1;   // fused FP32 transfer with the velocity box staged in shared memory
    int tuned = 0;
    cudaStream_t aux[2] = {};   // fork-join streams of ifem_step_coupling
    static constexpr int kForkEvents = 10;
    cudaEvent_t fork[kForkEvents] = {};
};

struct ifem_tmpl_s {
    ifem_ctx ctx;
    int kind;  // 0 membrane, 1 solid
    int law;
    int n_nodes, n_elems;
    double mu, C, kb, c0, lam;
    int *d_elems = nullptr;
    double *d_ref_d = nullptr;
    float *d_ref_f = nullptr;
    int *d_inc_off = nullptr;
    int *d_inc_idx = nullptr;
    int2 *d_ring = nullptr;
};

struct ifem_grid_s {
    ifem_ctx ctx;
    int n_boxes;
    std::vector<int> n;
    std::vector<double> L;
    std::vector<long long> off;
    long long total;
};

struct Workspace {
    ifem_grid grid = nullptr;
    int tile = 0;
    long long n_tiles = 0;
    int max_edge = 0;
    BoxDev *d_boxes = nullptr;
    DevWork w{};
    std::vector<void *> allocs;
};

struct ifem_batch_s {
    ifem_ctx ctx;
    std::vector<ifem_tmpl> tmpls;
    std::vector<ifem_instance_desc> inst;
    std::vector<InstDev> h_inst;
    long long N = 0;
    long long n_elems = 0;
    int max_nodes = 0, max_elems = 0;
    int any_bending = 0, fused_ok = 0;
    int max_box = 0;
    ifem_grid grid0 = nullptr;
    InstDev *d_inst = nullptr;
    TmplDev *d_tmpl = nullptr;
    int *d_node_inst = nullptr;
    void *d_elem_buf = nullptr;
    void *d_bend_buf = nullptr;
    Workspace ws;
};

// Makes `dev` the calling thread's current device for the lifetime of the
// object and then gives the caller's previous current device back, so that an
// entry point leaves the caller's device selection as it found it (dev < 0:
// nothing to do). The entry points' own cudaSetDevice calls inside the scope
// select the same device again.
struct DeviceScope {
    int prev = -1, dev = -1;
    explicit DeviceScope(int d) : dev(d)
    {
        if (dev < 0)
            return;
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        if (prev != dev)
            cudaSetDevice(dev);
    }
    ~DeviceScope()
    {
        if (dev >= 0 && prev >= 0 && prev != dev)
            cudaSetDevice(prev);
    }
    DeviceScope(const DeviceScope &) = delete;
    DeviceScope &operator=(const DeviceScope &) = delete;
};
#define IFEM_DEVICE_SCOPE(c) DeviceScope ifem_device_scope_((c) ? (c)->cfg.device : -1)

inline DevBatch dev_batch(ifem_batch b)
{
    DevBatch d{};
    d.n_inst = (int)b->inst.size();
    d.n_tmpl = (int)b->tmpls.size();
    d.N = b->N;
    d.max_nodes = b->max_nodes;
    d.max_elems = b->max_elems;
    d.n_elems_total = b->n_elems;
    d.any_bending = b->any_bending;
    d.fused_ok = b->fused_ok;
    d.inst = b->d_inst;
    d.tmpl = b->d_tmpl;
    d.node_inst = b->d_node_inst;
    return d;
}

