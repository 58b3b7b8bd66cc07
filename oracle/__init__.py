"""FP64 CPU oracle of the standard ALIF model -- test infrastructure only.

Only tests/, the smoke check and the bench's CPU-baseline leg may import this
package.  The CUDA product path never touches it.
"""
