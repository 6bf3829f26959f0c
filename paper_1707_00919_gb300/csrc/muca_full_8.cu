// muca_full_8.cu - whole-sweep kernels for L = 8.
#define MUCA_L 8
#include "muca_full.cuh"
