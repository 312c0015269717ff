// launch.cuh -- launch bookkeeping shared by the residual and adjoint
// kernels: every launch is counted, and timed when the scheme's timer is on.
#pragma once

#include <cuda_runtime.h>

#include "hfv_internal.h"

namespace hfv {

// scope guard: counts the launch and, when the scheme's timer is on, brackets
// it with a pair of events on the launch stream
struct Launch {
    KernelTimer* t;
    cudaStream_t st;
    int pair = -1;
    Launch(hfv_scheme* s, int kid, cudaStream_t stream) : t(&s->timer), st(stream)
    {
        note_launch();
        if (t->on && 2 * (t->used + 1) <= (int)t->ev.size()) {
            pair = t->used++;
            t->kid[pair] = kid;
            cudaEventRecord((cudaEvent_t)t->ev[2 * pair], st);
        }
    }
    ~Launch()
    {
        if (pair >= 0) cudaEventRecord((cudaEvent_t)t->ev[2 * pair + 1], st);
    }
};

}  // namespace hfv
