"""FP64 CPU oracle for the CutQC reconstruction path.

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously-correct numpy code that
restates what the paper defines.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import it; the library never does, and this
package imports nothing from the library.

Modules:
* ``statevector``  brute-force simulation of the uncut circuit (ground truth,
                   Background section: state-vector simulation).
* ``attribution``  subcircuit variants -> edge-basis tensors (the Pauli
                   decomposition behind Circuit Cutting, Eq. 1).
* ``fd``           full-definition reconstruction, Eq. 1 term by term.
* ``dd``           dynamic-definition query, Algorithm 1.
* ``metrics``      total variation, chi^2 (Eq. 3), normalisation error.
* ``mlp``          float64 forward/backward/Adam of the cut-scoring MLP.

Parity notes: every function names its pin in the tests; functions without a
pin say "parity unpinned" in their docstring (none at present).
"""
