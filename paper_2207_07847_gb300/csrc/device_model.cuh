// Device-resident model and workspaces of one solver handle.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <vector>

#include "kernels.cuh"
#include "lap_internal.h"

namespace lap {

// RAII device buffer from the library allocator.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { reset(); }
    void reset()
    {
        if (p) dev_free(p, nullptr);
        p = nullptr;
        bytes = 0;
    }
    bool alloc(size_t b)
    {
        reset();
        if (b == 0) b = 16;
        p = dev_alloc(b, nullptr);
        bytes = p ? b : 0;
        return p != nullptr;
    }
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

template <typename V> struct DevCsr {
    int n = 0;
    int64_t nnz = 0;
    int *rp = nullptr, *ci = nullptr;
    V *w = nullptr, *dg = nullptr;
};

template <typename V> struct DevMspLevel {
    int n = 0, nagg = 0;
    int64_t off = 0;            // expanded offset of this level (tree order)
    int *seg = nullptr;         // shared between precisions
    V *inv = nullptr, *lcf = nullptr;
};

template <typename V> struct DevMsp {
    int levels = 0;
    std::vector<DevMspLevel<V>> lev;   // levels 1..l-1 (index k-1)
    std::vector<int64_t> off;          // expanded offsets, size l+1
    std::vector<V> gamma;              // c_{k+1} / c_k per level k < l
    std::vector<double> c;             // c_k = sum_{i<k} (-mu)^i per level (index k-1)
    double *G = nullptr;               // dense top-level pseudo-inverse (FP64)
    int ntop = 0;
    V mu = V(0);
};

// Reduction scratch + device scalars of one CG.
struct CgState {
    CgScalars *sc = nullptr;
    double *part = nullptr;
    unsigned *ticket = nullptr;
};

// Vectors of one CG on L (n-space), preconditioned by the sweeps.
template <typename V> struct CgVectors {
    V *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr;
    V *A = nullptr, *Y = nullptr, *T = nullptr;   // expanded-space sweep buffers (ntilde)
};

}  // namespace lap
