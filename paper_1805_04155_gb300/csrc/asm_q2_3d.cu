// Hot-path kernels instantiated for the Q2_3D element (one translation unit per
// element type keeps the build parallel).
#include "assemble.cuh"

EP_DEFINE_ELEM_LAUNCHERS(7)
