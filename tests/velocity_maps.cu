// Prints the velocity index maps of the CUDA library (host side of its constexpr
// functions): for each velocity i, its x and y direction signs, the velocity whose
// value it holds on a y-symmetric state, and the mirror plane a computed velocity
// also writes (-1: none).  Then the distinct velocities in the order the symmetric
// kernels compute them.
#include <cstdio>

#include "cdbm_device.cuh"

int main()
{
    for (int i = 0; i < cdbm::kNV; ++i)
        std::printf("%d %d %d %d %d\n", i, cdbm::dirx(i), cdbm::diry(i), cdbm::mirror_y(i), cdbm::sym_partner(i));
    for (int k = 0; k < cdbm::kNSym; ++k) std::printf("%d ", cdbm::sym_vel(k));
    std::printf("\n");
    return 0;
}
