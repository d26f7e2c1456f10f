// dense_md_f16.cu -- the persistent tcgen05 dense MD kernel instantiated for
// the FP16 operand (HQA_PREC_FP16, HQA_PREC_FP16X2).  Kept apart from the BF16
// instantiations in dense_md.cu so that the two compile in parallel.
#include "dense_md_kernel.cuh"

template hqa_status hqa_dense::dense_md_dispatch<true>(hqa_ctx*, const hqa_dense::DenseMDArgs&,
                                                       int, int, int, cudaStream_t,
                                                       const CUtensorMap&, const CUtensorMap&,
                                                       const CUtensorMap&);
