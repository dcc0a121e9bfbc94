// Instantiations of the face sweep for the twelve-point TENO-AA scheme (S6 derived
// by the Sec. 4.1 recipe, see teno_coeffs.cuh).
#include "teno_face.cuh"

namespace teno {

cudaError_t launch_face12(int nd, int d, const FaceArgs &a, cudaStream_t s)
{
    switch (nd * 3 + d) {
    case 3: return launch_face<1, 6, 0>(a, s);
    case 6: return launch_face<2, 6, 0>(a, s);
    case 7: return launch_face<2, 6, 1>(a, s);
    case 9: return launch_face<3, 6, 0>(a, s);
    case 10: return launch_face<3, 6, 1>(a, s);
    case 11: return launch_face<3, 6, 2>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace teno
