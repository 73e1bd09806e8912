/*
 * pm_limits.h -- size limits of the confidence-aware human prediction
 * library (included by pm.h; the device code includes only this file).
 */
#ifndef PM_LIMITS_H_
#define PM_LIMITS_H_

#define PM_MAX_HEADINGS 64    /* K in [1, 64]                      */
#define PM_MAX_COMPONENTS 256 /* G*B in [1, 256]                   */
#define PM_MAX_GOALS 64       /* G in [1, 64]                      */
#define PM_MAX_HORIZON 4096   /* T in [1, 4096]                    */
#define PM_MAX_SPEEDS 4       /* speeds of the control set         */

#endif /* PM_LIMITS_H_ */
