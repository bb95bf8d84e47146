// fp64tc_blocks.cu -- the FP64 factorization on the tensor cores at tile
// orders 128 r, r > 1 (a task runs its r x r blocks of order 128 in the order
// of tile order 128): the launches of that instantiation of the task body,
// in a translation unit of their own (it compiles in parallel with fp64tc.cu).
#include "fp64tc_body.cuh"

namespace chol {

int fp64tc_launch_blocks(const OzArgs &g, const SchedArgs &a, const DFArgs *d, int Ml, int variant,
                         const chol_opts &o, cudaStream_t st, int *launches, cudaEvent_t e0) {
    if (d) return launch_dataflow<OzBodyBlocks>(g, a, *d, o, st, launches, e0);
    return run_fork_join<OzBodyBlocks>(g, a, Ml, variant, st, launches, e0, o.timeout_s);
}

}  // namespace chol
