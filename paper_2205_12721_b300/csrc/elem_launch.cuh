// Launch helpers shared by the element-kernel translation units.
#pragma once

#include "elem_kernels.cuh"
#include "tmop_internal.h"

namespace tmop {

template <class K>
static inline cudaError_t prepare(K kernel, size_t smem_bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

template <class C>
static inline int64_t grid_of(int64_t E)
{
    return (E + C::EPB - 1) / C::EPB;
}

}  // namespace tmop

#define TMOP_SWITCH(d, p, q, CALL)                                 \
    switch (TMOP_KEY(d, p, q)) {                                   \
        TMOP_CONFIGS(CALL)                                         \
        default: return cudaErrorInvalidValue;                     \
    }
