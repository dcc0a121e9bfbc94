// Instantiations of the face sweep for the 8-point TENO-AA scheme.
#include "teno_face.cuh"

namespace teno {

cudaError_t launch_face8(int nd, int d, const FaceArgs &a, cudaStream_t s)
{
    switch (nd * 3 + d) {
    case 3: return launch_face<1, 4, 0>(a, s);
    case 6: return launch_face<2, 4, 0>(a, s);
    case 7: return launch_face<2, 4, 1>(a, s);
    case 9: return launch_face<3, 4, 0>(a, s);
    case 10: return launch_face<3, 4, 1>(a, s);
    case 11: return launch_face<3, 4, 2>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace teno
