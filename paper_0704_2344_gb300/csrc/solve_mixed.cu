// Instantiates the persistent solve kernels (single system and jobs) for
// complex64 products with FP32 accumulation; one translation unit per product arithmetic.
#include "solve_kernels.cuh"

namespace fe {
template fe_status dispatch<float>(fe_ctx*, int, SolveParams&);
template fe_status launch_jobs_w<float>(fe_ctx*, int, SolveJob* const*, const int*, int, cudaStream_t, const int*);
}  // namespace fe
