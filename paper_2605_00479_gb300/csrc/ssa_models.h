// ssa_models.h -- reaction-network structures with compiled-in kernels.
//
// A model passed to ssa_model_create whose structure (species count,
// reactant orders, change vectors, laws, Hill exponents and regulators,
// constant species) equals one of these runs on a kernel with the structure
// fixed at compile time; rate constants, initial state and Hill amplitudes
// stay runtime values.  Any other model runs on the general kernel.
// The five structures are the paper's test systems (Sec. 4.1-4.5).
#pragma once

namespace ssa {
namespace models {

// 0 -> X, X -> 0 (Sec. 4.1)
struct BirthDeath {
    static constexpr int family = 1, N = 1, M = 2;
    static constexpr int ord[M][N] = {{0}, {1}};
    static constexpr int nu[M][N] = {{1}, {-1}};
    static constexpr int lw[M] = {0, 0};
    static constexpr int hh[M] = {0, 0};
    static constexpr int hreg[M] = {0, 0};
    static constexpr int cs[N] = {0};
};

// species (X, A, B); A + 2X <-> 3X, B <-> X; A and B held fixed (Sec. 4.2)
struct Schlogl {
    static constexpr int family = 2, N = 3, M = 4;
    static constexpr int ord[M][N] = {{2, 1, 0}, {3, 0, 0}, {0, 0, 1}, {1, 0, 0}};
    static constexpr int nu[M][N] = {{1, -1, 0}, {-1, 1, 0}, {1, 0, -1}, {-1, 0, 1}};
    static constexpr int lw[M] = {0, 0, 0, 0};
    static constexpr int hh[M] = {0, 0, 0, 0};
    static constexpr int hreg[M] = {0, 0, 0, 0};
    static constexpr int cs[N] = {0, 1, 1};
};

// species (Goff, Gon, M) (Sec. 4.3)
struct Telegraph {
    static constexpr int family = 3, N = 3, M = 4;
    static constexpr int ord[M][N] = {{1, 0, 0}, {0, 1, 0}, {0, 1, 0}, {0, 0, 1}};
    static constexpr int nu[M][N] = {{-1, 1, 0}, {1, -1, 0}, {0, 0, 1}, {0, 0, -1}};
    static constexpr int lw[M] = {0, 0, 0, 0};
    static constexpr int hh[M] = {0, 0, 0, 0};
    static constexpr int hreg[M] = {0, 0, 0, 0};
    static constexpr int cs[N] = {0, 0, 0};
};

// species (M, D); 2M <-> D (Sec. 4.4)
struct Dimer {
    static constexpr int family = 4, N = 2, M = 2;
    static constexpr int ord[M][N] = {{2, 0}, {0, 1}};
    static constexpr int nu[M][N] = {{-2, 1}, {2, -1}};
    static constexpr int lw[M] = {0, 0};
    static constexpr int hh[M] = {0, 0};
    static constexpr int hreg[M] = {0, 0};
    static constexpr int cs[N] = {0, 0};
};

// species (MA, MB, MC, PA, PB, PC); per gene: Hill transcription (h = 2,
// repressors C, A, B), mRNA decay, translation, protein decay (Sec. 4.5)
struct Repressilator {
    static constexpr int family = 5, N = 6, M = 12;
    static constexpr int ord[M][N] = {
        {0, 0, 0, 0, 0, 0}, {1, 0, 0, 0, 0, 0}, {1, 0, 0, 0, 0, 0}, {0, 0, 0, 1, 0, 0},
        {0, 0, 0, 0, 0, 0}, {0, 1, 0, 0, 0, 0}, {0, 1, 0, 0, 0, 0}, {0, 0, 0, 0, 1, 0},
        {0, 0, 0, 0, 0, 0}, {0, 0, 1, 0, 0, 0}, {0, 0, 1, 0, 0, 0}, {0, 0, 0, 0, 0, 1}};
    static constexpr int nu[M][N] = {
        {1, 0, 0, 0, 0, 0}, {-1, 0, 0, 0, 0, 0}, {0, 0, 0, 1, 0, 0}, {0, 0, 0, -1, 0, 0},
        {0, 1, 0, 0, 0, 0}, {0, -1, 0, 0, 0, 0}, {0, 0, 0, 0, 1, 0}, {0, 0, 0, 0, -1, 0},
        {0, 0, 1, 0, 0, 0}, {0, 0, -1, 0, 0, 0}, {0, 0, 0, 0, 0, 1}, {0, 0, 0, 0, 0, -1}};
    static constexpr int lw[M] = {1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0};
    static constexpr int hh[M] = {2, 0, 0, 0, 2, 0, 0, 0, 2, 0, 0, 0};
    static constexpr int hreg[M] = {5, 0, 0, 0, 3, 0, 0, 0, 4, 0, 0, 0};
    static constexpr int cs[N] = {0, 0, 0, 0, 0, 0};
};

}  // namespace models
}  // namespace ssa
