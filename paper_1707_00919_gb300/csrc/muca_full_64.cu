// muca_full_64.cu - whole-sweep kernels for L = 64.
#define MUCA_L 64
#include "muca_full.cuh"
