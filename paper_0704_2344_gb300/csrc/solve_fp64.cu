// Instantiates the persistent solve kernels (single system and jobs) for
// complex128 products on the FP64 pipes; one translation unit per product arithmetic.
#include "solve_kernels.cuh"

namespace fe {
template fe_status dispatch<double>(fe_ctx*, int, SolveParams&);
template fe_status launch_jobs_w<double>(fe_ctx*, int, SolveJob* const*, const int*, int, cudaStream_t, const int*);
}  // namespace fe
