"""FP64 CPU oracle of the CAC-LB wetting step -- TEST INFRASTRUCTURE.

Only tests, the smoke check and the bench's CPU-baseline leg may import this
package. The product path never loads it.
"""
