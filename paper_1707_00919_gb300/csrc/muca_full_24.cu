// muca_full_24.cu - whole-sweep kernels for L = 24.
#define MUCA_L 24
#include "muca_full.cuh"
