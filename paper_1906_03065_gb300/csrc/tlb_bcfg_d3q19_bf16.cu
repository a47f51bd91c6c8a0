// Instantiation of the batched driver for one velocity set and storage precision.
#include "tlb_batch.cuh"

static_assert(sizeof(BArgs<TLB_BF16>) <= Batch::ARGS_BYTES, "instance argument record too large");

BatchBase* make_batch_impl_d3q19_bf16() {
  static BatchImpl<D3Q19, TLB_BF16> impl;
  return &impl;
}
