// Persistent batched kernels for element orders 7, 8 and 9 (the orders are
// spread over three translation units so that they compile in parallel).
#include "batch_kernel.cuh"

namespace femfft {

const void* batch_kernel_fn_3(int n) {
  switch (n) {
    case 7: return (const void*)batch_kernel<7>;
    case 8: return (const void*)batch_kernel<8>;
    case 9: return (const void*)batch_kernel<9>;
    default: return nullptr;
  }
}

}  // namespace femfft
