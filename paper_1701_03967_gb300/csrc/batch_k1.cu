// Persistent batched kernels for element orders 1, 2 and 3 (the orders are
// spread over three translation units so that they compile in parallel).
#include "batch_kernel.cuh"

namespace femfft {

const void* batch_kernel_fn_1(int n) {
  switch (n) {
    case 1: return (const void*)batch_kernel<1>;
    case 2: return (const void*)batch_kernel<2>;
    case 3: return (const void*)batch_kernel<3>;
    default: return nullptr;
  }
}

}  // namespace femfft
