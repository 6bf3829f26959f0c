// muca_full_16.cu - whole-sweep kernels for L = 16.
#define MUCA_L 16
#include "muca_full.cuh"
