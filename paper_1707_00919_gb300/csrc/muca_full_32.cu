// muca_full_32.cu - whole-sweep kernels for L = 32.
#define MUCA_L 32
#include "muca_full.cuh"
