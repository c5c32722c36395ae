// Persistent batched kernels for element orders 4, 5 and 6 (the orders are
// spread over three translation units so that they compile in parallel).
#include "batch_kernel.cuh"

namespace femfft {

const void* batch_kernel_fn_2(int n) {
  switch (n) {
    case 4: return (const void*)batch_kernel<4>;
    case 5: return (const void*)batch_kernel<5>;
    case 6: return (const void*)batch_kernel<6>;
    default: return nullptr;
  }
}

}  // namespace femfft
