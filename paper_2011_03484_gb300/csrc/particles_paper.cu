// particles_paper.cu -- the test-particle map with the paper's fixed-iteration
// Kepler solve (section 2.2; GLISSE_KEPLER_PAPER_FIXED), in its own translation
// unit so that it compiles in parallel with the default kernels.
#include "particle_map.cuh"

namespace glisse {

cudaError_t launch_particle_chunk_paper(int np, const ChunkArgs& a, const ParticleConsts& pc, cudaStream_t s) {
    return launch_particle_chunk_mode<kDriftPaper>(np, a, pc, s);
}

}  // namespace glisse
