"""FP64 CPU oracle for the GP-BO hot path -- test infrastructure only.

Only the tests, the smoke check and the bench's CPU-baseline leg import this
package.  The product library never loads it.
"""
